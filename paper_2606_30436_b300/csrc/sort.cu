// sort.cu -- binning of projected Gaussians into (tile, depth)-ordered pairs.
//
// The order required is that of a stable sort by the 64-bit key
// (global tile << 32) | depth bits with ties broken by record index ("sorted
// Gaussians along the ray", Supp. D.2).  It is produced in two cheaper stages:
//   1. the visible records (radius > 0), compacted in index order, are sorted
//      once by their 32-bit depth with a stable LSD radix sort, giving each a
//      depth rank;
//   2. every visible record emits one (tile, rank) pair per overlapped tile,
//      in rank order, and a stable LSD radix sort on the tile bits alone puts
//      the pairs in tile order while keeping rank order inside a tile.
// Stage 2 moves 8 bytes per pair over ceil(tile_bits / 8) passes instead of
// 12 bytes over ceil((32 + tile_bits) / 8) passes for the 64-bit key.
// Every kernel reads its element count from device memory and runs on a fixed
// grid, so the sequence needs no host synchronisation and can be captured.
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
    __shared__ unsigned long long sm[33];
    long long beg, end;
    block_segment(nrec, beg, end);
    unsigned long long c = 0;
    for (long long i = beg + threadIdx.x; i < end; i += kSortThreads) c += radius[i] > 0;
    unsigned long long total;
    block_exclusive_scan<unsigned long long>(c, total, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// Exclusive scan of the per-block sums (one block of kSortBlocks threads).
// mode 0: total -> counts[0] (visible records).
// mode 1: total -> pairs; counts[2] = needed, counts[1] = pairs or 0 on overflow.
__global__ void __launch_bounds__(kSortBlocks) k_scan_blocks(unsigned long long *__restrict__ blk, int mode,
                                                             int *__restrict__ counts, long long max_pairs,
                                                             int *__restrict__ status) {
    __shared__ unsigned long long sm[33];
    unsigned long long x = blk[threadIdx.x], total;
    unsigned long long ex = block_exclusive_scan<unsigned long long>(x, total, sm);
    blk[threadIdx.x] = ex;
    if (threadIdx.x == 0) {
        const int t32 = (int)min(total, (unsigned long long)0x7fffffff);
        if (mode == 0) {
            counts[0] = t32;
        } else {
            counts[2] = t32;
            const bool ok = total <= (unsigned long long)max_pairs;
            counts[1] = ok ? t32 : 0;
            if (!ok && status) atomicOr(status, 1 << GS_ERR_CAPACITY);
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_visible_compact(const int *__restrict__ radius,
                                                                   const float4 *__restrict__ rgbd, long long nrec,
                                                                   const unsigned long long *__restrict__ blk,
                                                                   uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    __shared__ unsigned long long sm[33];
    long long beg, end;
    block_segment(nrec, beg, end);
    unsigned long long run = blk[blockIdx.x];
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
// stable LSD radix sort pass (keys u32 with u32 values), digit of `bits` <= 8
// bits at `shift`; element count read from *count.

__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                 const int *__restrict__ count, int shift, int bits,
                                                                 uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    const int radix = 1 << bits;
    const uint32_t mask = radix - 1;
    for (int i = threadIdx.x; i < radix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const long long cnt_all = *count;
    const long long seg = ceil_div(ceil_div(cnt_all, (long long)gridDim.x), (long long)(kSortThreads * 16)) *
                          (kSortThreads * 16);  // same segments as the downsweep (kDownTile)
    const long long beg = min(cnt_all, (long long)blockIdx.x * seg), end = min(cnt_all, beg + seg);
    for (long long i = beg + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kSortThreads) hist[d * kSortBlocks + blockIdx.x] = h[d];
}

// One block per digit: exclusive scan of the digit's per-block counts.
__global__ void __launch_bounds__(kSortBlocks) k_radix_scan(uint32_t *__restrict__ hist, uint32_t *__restrict__ dtotal) {
    __shared__ uint32_t sm[33];
    const int d = blockIdx.x;
    uint32_t x = hist[d * kSortBlocks + threadIdx.x], total;
    uint32_t ex = block_exclusive_scan<uint32_t>(x, total, sm);
    hist[d * kSortBlocks + threadIdx.x] = ex;
    if (threadIdx.x == 0) dtotal[d] = total;
}

// Stable scatter of one LSD pass.  A block takes its segment in rounds of
// kDownTile elements; each warp ranks its 512 consecutive elements (16 rounds
// of 32 lanes) per digit with ballots (lanes whose digit bits all agree) and
// a per-warp histogram, the warps' counts are scanned per digit, the round is
// reordered by digit in shared memory, and written out in digit runs so that
// the global stores are contiguous.
constexpr int kDownItems = 16;
constexpr int kDownTile = kSortThreads * kDownItems;  // 4096

// With `rec` set (the last pass of the pair sort; only tested for null), the
// scatter writes the outputs the renderer reads instead of the raw pairs: the
// record (the pair's value) into vout, the block mask (key >> 24) into masks,
// and the tile (key & 0xffffff) into kout for the range pass.
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_downsweep(const uint32_t *__restrict__ kin,
                                                                   const uint32_t *__restrict__ vin,
                                                                   uint32_t *__restrict__ kout,
                                                                   uint32_t *__restrict__ vout,
                                                                   const int *__restrict__ count, int shift, int bits,
                                                                   const uint32_t *__restrict__ hist,
                                                                   const uint32_t *__restrict__ dtotal,
                                                                   const uint32_t *__restrict__ rec,
                                                                   uint8_t *__restrict__ masks) {
    __shared__ uint32_t s_base[256];    // global position of this block's next element of each digit
    __shared__ uint32_t s_dstart[256];  // first local slot of each digit in the current round
    __shared__ uint32_t s_whist[kSortThreads / 32][256];
    __shared__ uint32_t s_key[kDownTile];
    __shared__ uint32_t s_val[kDownTile];
    __shared__ uint32_t sm[33];
    const int radix = 1 << bits;
    const uint32_t mask = radix - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;

    {
        uint32_t t = threadIdx.x < radix ? dtotal[threadIdx.x] : 0u, tot;
        uint32_t ex = block_exclusive_scan<uint32_t>(t, tot, sm);
        if (threadIdx.x < radix) s_base[threadIdx.x] = ex + hist[threadIdx.x * kSortBlocks + blockIdx.x];
    }
    __syncthreads();
    const long long cnt_all = *count;
    const long long seg = ceil_div(ceil_div(cnt_all, (long long)gridDim.x), (long long)kDownTile) * kDownTile;
    const long long beg = min(cnt_all, (long long)blockIdx.x * seg), end = min(cnt_all, beg + seg);
    for (long long tb = beg; tb < end; tb += kDownTile) {
        for (int i = lane; i < radix; i += 32) s_whist[warp][i] = 0;
        __syncwarp();
        uint32_t k[kDownItems], v[kDownItems], rk[kDownItems];
        #pragma unroll
        for (int r = 0; r < kDownItems; ++r) {
            const long long idx = tb + warp * (32 * kDownItems) + r * 32 + lane;
            const bool valid = idx < end;
            k[r] = valid ? kin[idx] : 0xffffffffu;
            v[r] = valid ? vin[idx] : 0u;
        }
        #pragma unroll
        for (int r = 0; r < kDownItems; ++r) {
            const long long idx = tb + warp * (32 * kDownItems) + r * 32 + lane;
            const bool valid = idx < end;
            const uint32_t d = (k[r] >> shift) & mask;
            // lanes holding the same digit: all `bits` ballots agree
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            for (int b = 0; b < bits; ++b) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            uint32_t base = 0;
            const int leader = __ffs(peers) - 1;
            if (valid && lane == leader) {
                base = s_whist[warp][d];
                s_whist[warp][d] = base + __popc(peers);
            }
            base = __shfl_sync(0xffffffffu, base, valid ? leader : 0);
            rk[r] = valid ? base + __popc(peers & lt) : 0xffffffffu;
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive scan over warps, and the round's digit totals
        for (int dd = threadIdx.x; dd < radix; dd += kSortThreads) {
            uint32_t sacc = 0;
            #pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = s_whist[w][dd];
                s_whist[w][dd] = sacc;
                sacc += c;
            }
            s_dstart[dd] = sacc;  // round total of digit dd (scanned below)
        }
        __syncthreads();
        {
            uint32_t t = threadIdx.x < radix ? s_dstart[threadIdx.x] : 0u, tot;
            const uint32_t ex = block_exclusive_scan<uint32_t>(t, tot, sm);
            if (threadIdx.x < radix) s_dstart[threadIdx.x] = ex;
        }
        __syncthreads();
        // reorder the round by digit in shared memory
        #pragma unroll
        for (int r = 0; r < kDownItems; ++r) {
            if (rk[r] != 0xffffffffu) {
                const uint32_t d = (k[r] >> shift) & mask;
                const uint32_t slot = s_dstart[d] + s_whist[warp][d] + rk[r];
                s_key[slot] = k[r];
                s_val[slot] = v[r];
            }
        }
        __syncthreads();
        const int n_round = (int)min((long long)kDownTile, end - tb);
        if (rec) {
            for (int i = threadIdx.x; i < n_round; i += kSortThreads) {
                const uint32_t key = s_key[i];
                const uint32_t d = (key >> shift) & mask;
                const uint32_t pos = s_base[d] + (uint32_t)i - s_dstart[d];
                kout[pos] = key & 0xffffffu;
                vout[pos] = s_val[i];  // the record
                masks[pos] = (uint8_t)(key >> 24);
            }
        } else {
            for (int i = threadIdx.x; i < n_round; i += kSortThreads) {
                const uint32_t key = s_key[i];
                const uint32_t d = (key >> shift) & mask;
                const uint32_t pos = s_base[d] + (uint32_t)i - s_dstart[d];
                kout[pos] = key;
                vout[pos] = s_val[i];
            }
        }
        __syncthreads();
        // advance the block's digit bases by this round's counts
        for (int dd = threadIdx.x; dd < radix; dd += kSortThreads) {
            const uint32_t nxt = (dd + 1 < radix) ? s_dstart[dd + 1] : (uint32_t)n_round;
            s_base[dd] += nxt - s_dstart[dd];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// stage 2: pair emission in depth-rank order

__global__ void __launch_bounds__(kSortThreads) k_tiles_count(const uint32_t *__restrict__ sorted_rec,
                                                               const int *__restrict__ touched,
                                                               const int *__restrict__ counts,
                                                               unsigned long long *__restrict__ blk) {
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
                                                                 uint32_t *__restrict__ off) {
    __shared__ unsigned long long sm[33];
    const long long V = counts[0];
    long long beg, end;
    block_segment(V, beg, end);
    unsigned long long run = blk[blockIdx.x];
    for (long long base = beg; base < end; base += kSortThreads) {
        const long long r = base + threadIdx.x;
        const int tt = r < end ? touched[sorted_rec[r]] : 0;
        unsigned long long total;
        const unsigned long long o = run + block_exclusive_scan<unsigned long long>((unsigned long long)tt, total, sm);
        if (r < end) off[r] = (uint32_t)o;
        run += total;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[V] = (uint32_t)counts[2];
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

// Tile ranges from the sorted tile keys (the last sort pass already wrote
// the Gaussian ids and block masks).
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *__restrict__ tkey, const int *__restrict__ counts,
                                                 int2 *__restrict__ ranges) {
    const long long P = counts[1];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = tkey[p];
        if (p == 0 || tkey[p - 1] != t) ranges[t].x = (int)p;
        if (p == P - 1 || tkey[p + 1] != t) ranges[t].y = (int)(p + 1);
    }
}

// Without a tile pass (one tile in all): ids and masks straight from the
// emitted pairs, which are already in order.
__global__ void __launch_bounds__(256) k_unpack_pairs(const uint32_t *__restrict__ pkey,
                                                       const uint32_t *__restrict__ pval,
                                                       const uint32_t *__restrict__ rec, const int *__restrict__ counts,
                                                       uint32_t *__restrict__ tkey, int *__restrict__ ids,
                                                       uint8_t *__restrict__ masks) {
    const long long P = counts[1];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t key = pkey[p];
        tkey[p] = key & 0xffffffu;
        ids[p] = (int)pval[p];
        masks[p] = (uint8_t)(key >> 24);
    }
}

// ---------------------------------------------------------------------------
// render schedule: tiles by descending pair count (log2 buckets), so the
// compositing kernels start the longest tiles first and their chains overlap
// the many short tiles instead of trailing them.

__global__ void __launch_bounds__(256) k_tile_hist(const int2 *__restrict__ ranges, int total_tiles,
                                                    unsigned int *__restrict__ bucket) {
    __shared__ unsigned int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        const int2 r = ranges[t];
        const unsigned c = (unsigned)(r.y - r.x);
        atomicAdd(&h[c ? 32 - __clz(c) : 0], 1u);  // 0 for empty, 1 + floor(log2 c) otherwise
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&bucket[threadIdx.x], h[threadIdx.x]);
}

// cursors: bucket 32 (longest) first
__global__ void k_tile_scan(unsigned int *__restrict__ bucket) {
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int b = 32; b >= 0; --b) {
            const unsigned int c = bucket[b];
            bucket[b] = run;
            run += c;
        }
    }
}

__global__ void __launch_bounds__(256) k_tile_scatter(const int2 *__restrict__ ranges, int total_tiles,
                                                       unsigned int *__restrict__ bucket, int *__restrict__ order) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        const int2 r = ranges[t];
        const unsigned c = (unsigned)(r.y - r.x);
        order[atomicAdd(&bucket[c ? 32 - __clz(c) : 0], 1u)] = t;
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
    w.bucket = (unsigned int *)take(sizeof(unsigned int) * 64);
    w.hist = (uint32_t *)take(sizeof(uint32_t) * 256 * kSortBlocks);
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

// Sorts (k, v) in place-by-ping-pong over bits [0, total_bits); returns which
// buffer pair holds the result (0: k0/v0, 1: k1/v1).
// LSD radix sort of (k, v) on bits [0, total_bits) by ping-pong; returns the
// buffer pair holding the result (0: k0/v0, 1: k1/v1).  With `rec` set the
// last pass writes tile keys, ids = rec[v] and masks (see k_radix_downsweep),
// the ids into final_v when given.
static int radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int *count, int total_bits,
                      uint32_t *hist, uint32_t *dtotal, cudaStream_t s, const uint32_t *rec = nullptr,
                      uint8_t *masks = nullptr, uint32_t *final_v = nullptr) {
    if (total_bits <= 0) return 0;
    const int passes = (total_bits + 7) / 8;
    const int width = (total_bits + passes - 1) / passes;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * width;
        const int bits = min(width, total_bits - shift);
        uint32_t *ki = cur ? k1 : k0, *vi = cur ? v1 : v0, *ko = cur ? k0 : k1, *vo = cur ? v0 : v1;
        const bool last = p == passes - 1;
        if (last && final_v) vo = final_v;
        k_radix_upsweep<<<kSortBlocks, kSortThreads, 0, s>>>(ki, count, shift, bits, hist);
        k_radix_scan<<<1 << bits, kSortBlocks, 0, s>>>(hist, dtotal);
        k_radix_downsweep<<<kSortBlocks, kSortThreads, 0, s>>>(ki, vi, ko, vo, count, shift, bits, hist, dtotal,
                                                                last ? rec : nullptr, last ? masks : nullptr);
        cur ^= 1;
    }
    return cur;
}

cudaError_t launch_sort(const int *radius, const int *touched, const float2 *xy, const float4 *co, const float4 *rgbd,
                        long long nrec, long long ld, const ViewTable &vt, float alpha_min, int *gauss_ids,
                        int2 *tile_ranges, uint8_t *block_mask, int *tile_order, int *counts, long long max_pairs,
                        void *ws, int *status, cudaStream_t s) {
    SortWs w = carve(ws, nrec, max_pairs);
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)vt.total_tiles, s);
    if (e != cudaSuccess) return e;

    // stage 1: visible records sorted by depth
    k_visible_count<<<kSortBlocks, kSortThreads, 0, s>>>(radius, nrec, w.blk);
    k_scan_blocks<<<1, kSortBlocks, 0, s>>>(w.blk, 0, counts, max_pairs, status);
    k_visible_compact<<<kSortBlocks, kSortThreads, 0, s>>>(radius, rgbd, nrec, w.blk, w.dk0, w.dv0);
    const int dres = radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, counts + 0, 32, w.hist, w.dtotal, s);
    const uint32_t *sorted_rec = dres ? w.dv1 : w.dv0;

    // stage 2: pairs in rank order, then a stable partition by tile
    k_tiles_count<<<kSortBlocks, kSortThreads, 0, s>>>(sorted_rec, touched, counts, w.blk);
    k_scan_blocks<<<1, kSortBlocks, 0, s>>>(w.blk, 1, counts, max_pairs, status);
    k_tiles_offsets<<<kSortBlocks, kSortThreads, 0, s>>>(sorted_rec, touched, counts, w.blk, w.off);
    k_emit_pairs<<<148 * 16, 256, 0, s>>>(sorted_rec, w.off, radius, xy, co, ld, vt, alpha_min, counts, w.big, w.pk0,
                                          w.pv0);
    k_emit_big<<<148 * 4, 256, 0, s>>>(sorted_rec, w.off, radius, xy, co, ld, vt, alpha_min, counts, w.big, w.pk0,
                                       w.pv0);
    int tile_bits = 0;
    while ((1ll << tile_bits) < (long long)vt.total_tiles) ++tile_bits;
    const uint32_t *tkey;
    if (tile_bits > 0) {
        // the last pass writes tile keys and ids into the other buffer pair
        const int pres = radix_sort(w.pk0, w.pv0, w.pk1, w.pv1, counts + 1, tile_bits, w.hist, w.dtotal, s,
                                    sorted_rec, block_mask, (uint32_t *)gauss_ids);
        tkey = pres ? w.pk1 : w.pk0;
    } else {
        k_unpack_pairs<<<148 * 8, 256, 0, s>>>(w.pk0, w.pv0, sorted_rec, counts, w.pk1, gauss_ids, block_mask);
        tkey = w.pk1;
    }
    k_ranges<<<148 * 8, 256, 0, s>>>(tkey, counts, tile_ranges);
    e = cudaMemsetAsync(w.bucket, 0, sizeof(unsigned int) * 64, s);
    if (e != cudaSuccess) return e;
    const int tb = (int)std::min<long long>(ceil_div(vt.total_tiles, 256), 148 * 4);
    k_tile_hist<<<tb, 256, 0, s>>>(tile_ranges, vt.total_tiles, w.bucket);
    k_tile_scan<<<1, 32, 0, s>>>(w.bucket);
    k_tile_scatter<<<tb, 256, 0, s>>>(tile_ranges, vt.total_tiles, w.bucket, tile_order);
    return cudaGetLastError();
}

}  // namespace gs
