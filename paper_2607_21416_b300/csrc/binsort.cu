// binsort.cu -- (tile, depth) binning of splats and a stable LSD radix sort.
//
// Result order: (global tile, float bits of depth, splat id), i.e. the order
// of a sort on the 64-bit key (tile << 32 | depth bits) with ties broken by
// splat id.  It is reached without sorting 64-bit keys:
//   1. compact the splats that cover a tile (deterministic scan), keeping
//      candidate-id order;
//   2. stable radix sort of those splats on their 32-bit depth bits (ties
//      keep id order);
//   3. gather the splats' tile rectangles into depth order (once), scan
//      their tile counts (per-splat pair offsets) and emit
//      one (tile id, splat id) pair per covered tile, load-balanced: each
//      CTA round writes 2048 consecutive pairs; the scan also records the
//      splat that owns each round's first pair, and each pair finds its splat
//      by a max-scan over the round's staged first positions;
//   4. stable radix sort of the pairs on the tile id (only the bits the tile
//      count needs), which keeps depth-then-id order inside each tile;
//   5. tile ranges [start, end) and, on request, the 64-bit keys.
// Every size is read from device memory, so the sequence is graph-capturable.
#include "gs_internal.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 2048 elements
constexpr int kRadixItems = 8;                          // keys per thread of a radix pass tile
constexpr int kRadixTile = kSortThreads * kRadixItems;  // 2048 keys
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Tiles [t0, t1) of 2048 elements owned by block b of nb for n elements.
template <int TILE = kSortTile>
__device__ __forceinline__ void block_tiles(uint32_t n, int b, int nb, uint32_t *t0, uint32_t *t1)
{
    const uint32_t ntiles = (n + TILE - 1) / TILE;
    const uint32_t per = (ntiles + nb - 1) / nb;
    *t0 = min(ntiles, per * (uint32_t)b);
    *t1 = min(ntiles, per * (uint32_t)(b + 1));
}

// 256-thread block exclusive scan (returns exclusive prefix, writes total).
__device__ __forceinline__ uint32_t scan256(uint32_t x, uint32_t *s_warp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kSortWarps ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < kSortWarps; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kSortWarps) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t ex = v - x + (warp > 0 ? s_warp[warp - 1] : 0);
    *total = s_warp[kSortWarps - 1];
    __syncthreads();
    return ex;
}

// --------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const uint32_t *__restrict__ keys,
                                                              const uint32_t *__restrict__ n_ptr, int shift,
                                                              uint32_t *__restrict__ hist,
                                                              const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    __shared__ uint32_t s_h[kSortWarps * 256];   // per-warp histograms, flat
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) s_h[i] = 0;
    __syncthreads();
    const uint32_t n = *n_ptr;
    uint32_t t0, t1;
    block_tiles<kRadixTile>(n, blockIdx.x, gridDim.x, &t0, &t1);
    const int warp = threadIdx.x >> 5;
    const uint32_t e0 = t0 * kRadixTile, e1 = min(n, t1 * kRadixTile);
    // eight keys per thread per step, their loads issued together
    uint32_t i = e0 + threadIdx.x;
    for (; i + 7 * kSortThreads < e1; i += 8 * kSortThreads) {
        uint32_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) kk[j] = keys[i + j * kSortThreads];
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&s_h[warp * 256 + ((kk[j] >> shift) & 0xffu)], 1u);
    }
    for (; i < e1; i += kSortThreads) atomicAdd(&s_h[warp * 256 + ((keys[i] >> shift) & 0xffu)], 1u);
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) sum += s_h[w * 256 + threadIdx.x];
    hist[threadIdx.x * gridDim.x + blockIdx.x] = sum;
}

// One block per digit: exclusive scan of hist[d][0..nb) in place; totals[d].
__global__ void __launch_bounds__(1024) radix_scan_rows(uint32_t *__restrict__ hist, int nb,
                                                        uint32_t *__restrict__ totals, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    __shared__ uint32_t s_warp[32];
    const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = threadIdx.x < nb ? hist[d * nb + threadIdx.x] : 0;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t ex = v - x + (warp > 0 ? s_warp[warp - 1] : 0);
    if (threadIdx.x < nb) hist[d * nb + threadIdx.x] = ex;
    if (threadIdx.x == 0) totals[d] = s_warp[31];
}

// One scatter pass of the LSD radix sort (8-bit digit at `shift`), stable.
// kMatch: in-warp ranking by match_any, fast when a warp holds few distinct
// digits (the top digit of depth or tile keys); otherwise by one ballot per
// digit bit, whose cost does not depend on the digits.  kRanges (last pass of
// the tile sort): also records each tile's [start, end) in `ranges`, starts
// by atomicMin and ends by atomicMin of their complement (the array is set to
// all ones beforehand; finish_ranges turns untouched tiles into empty ones).
template <bool kMatch, bool kRanges>
__global__ void __launch_bounds__(kSortThreads, 4) radix_downsweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ n_ptr, int shift,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals, uint32_t *__restrict__ ranges,
    int n_ranges, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    __shared__ uint32_t s_keys[kRadixTile];
    __shared__ uint32_t s_vals[kRadixTile];
    // per-warp digit counts (then per-warp exclusive prefixes), flat
    // [warp][257]; column 256 collects the out-of-range lanes of a ragged tile
    __shared__ uint32_t s_wh[kSortWarps * 257];
    __shared__ uint32_t s_goff[256], s_tstart[256], s_tcnt[256];
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = *n_ptr;
    uint32_t t0, t1;
    block_tiles<kRadixTile>(n, blockIdx.x, gridDim.x, &t0, &t1);
    {   // global start of each digit for this block
        uint32_t tot;
        uint32_t pre = scan256(totals[tid], s_warp, &tot);
        s_goff[tid] = pre + hist[tid * gridDim.x + blockIdx.x];
    }
    for (int i = tid; i < kSortWarps * 257; i += kSortThreads) s_wh[i] = 0;
    __syncthreads();
    const unsigned ltm = lanemask_lt();
    // the next tile's keys and values are loaded while the current one is ranked and scattered
    uint32_t nkey[kRadixItems], nval[kRadixItems];
    auto load_tile = [&](uint32_t t) {
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            const uint32_t i = t * kRadixTile + warp * (32 * kRadixItems) + j * 32 + lane;
            nkey[j] = i < n ? kin[i] : 0u;
            nval[j] = i < n ? vin[i] : 0u;
        }
    };
    if (t0 < t1) load_tile(t0);
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t tb = t * kRadixTile;
        uint32_t key[kRadixItems], val[kRadixItems], loc[kRadixItems];
        int dig[kRadixItems];
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            const uint32_t i = tb + warp * (32 * kRadixItems) + j * 32 + lane;
            key[j] = nkey[j];
            val[j] = nval[j];
            dig[j] = i < n ? (int)((key[j] >> shift) & 0xffu) : 256;
        }
        if (t + 1 < t1) load_tile(t + 1);
        // Stable in-warp ranking, round by round: the lanes holding the same
        // digit are found from one ballot per digit bit (nine bits: 256 marks
        // an out-of-range lane), at a cost that does not depend on how many
        // distinct digits the warp holds; the lowest lane of each digit group
        // adds the group size to the warp's counter (shared-memory atomic,
        // returning the old count) and hands the old count to its peers.  Each
        // leader needs its atomic's result before the shuffle, so the rounds are
        // ordered by data dependence.
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            unsigned peers = 0xffffffffu;
            if (kMatch) {
                peers = __match_any_sync(0xffffffffu, dig[j]);
            } else {
#pragma unroll
                for (int bit = 0; bit < 9; ++bit) {
                    const bool set = (dig[j] >> bit) & 1;
                    const unsigned b = __ballot_sync(0xffffffffu, set);
                    peers &= set ? b : ~b;
                }
            }
            const int leader = __ffs(peers) - 1;
            const uint32_t rank = __popc(peers & ltm);
            uint32_t old = 0;
            if (rank == 0) old = atomicAdd(&s_wh[warp * 257 + dig[j]], (uint32_t)__popc(peers));
            old = __shfl_sync(0xffffffffu, old, leader);
            loc[j] = old + rank;
        }
        __syncthreads();
        {   // per digit: prefix over warps, tile count, tile-local start
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_wh[w * 257 + tid];
                s_wh[w * 257 + tid] = run;
                run += c;
            }
            s_tcnt[tid] = run;
            uint32_t tot;
            s_tstart[tid] = scan256(run, s_warp, &tot);
        }
        __syncthreads();   // s_tstart is written after the scan's last barrier
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            if (dig[j] < 256) {
                const uint32_t p = s_tstart[dig[j]] + s_wh[warp * 257 + dig[j]] + loc[j];
                if (!idx_ok(st, p, kRadixTile, 33)) continue;
                s_keys[p] = key[j];
                s_vals[p] = val[j];
            }
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kRadixTile, n - tb);
        for (uint32_t i = tid; i < cnt; i += kSortThreads) {
            const uint32_t k = s_keys[i];
            const uint32_t d = (k >> shift) & 0xffu;
            const uint32_t g = s_goff[d] + (i - s_tstart[d]);
            if (!idx_ok(st, g, n, 32)) continue;
            kout[g] = k;
            vout[g] = s_vals[i];
            if (kRanges) {   // equal keys are contiguous in the tile (ordered by the lower digits)
                if (!idx_ok(st, k, n_ranges, 38)) continue;
                if (i == 0 || s_keys[i - 1] != k) atomicMin(ranges + 2 * k, g);
                if (i + 1 == cnt || s_keys[i + 1] != k) atomicMin(ranges + 2 * k + 1, ~(g + 1));
            }
        }
        __syncthreads();
        s_goff[tid] += s_tcnt[tid];
        for (int i = tid; i < kSortWarps * 257; i += kSortThreads) s_wh[i] = 0;
        __syncthreads();
    }
}

// ------------------------------------------------------ compaction / emission
// Pass A of a two-pass scan over candidates: per-block count of covering splats.
__global__ void __launch_bounds__(kSortThreads) count_valid_kernel(
    const int32_t *__restrict__ tiles, const int32_t *__restrict__ view_start, int V, int k,
    long long cap_cand, uint32_t *__restrict__ block_sums, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t C = (uint32_t)min((long long)__ldg(view_start + V) * k, cap_cand);
    uint32_t t0, t1;
    block_tiles(C, blockIdx.x, gridDim.x, &t0, &t1);
    uint32_t n = 0;
    for (uint32_t i = t0 * kSortTile + threadIdx.x; i < min(C, t1 * kSortTile); i += kSortThreads)
        n += __ldg(tiles + i) > 0;
    __shared__ uint32_t s_warp[32];
    uint32_t tot;
    scan256(n, s_warp, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of nb block sums (nb <= 1024); total -> *out_n.
__global__ void __launch_bounds__(1024) scan_block_sums(uint32_t *__restrict__ sums, int nb,
                                                        uint32_t *__restrict__ out_n, long long cap,
                                                        gs_status *st, int where)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    __shared__ unsigned long long s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = threadIdx.x < nb ? sums[threadIdx.x] : 0ull;
    unsigned long long v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    unsigned long long ex = v - x + (warp > 0 ? s_warp[warp - 1] : 0ull);
    if (threadIdx.x < nb) sums[threadIdx.x] = (uint32_t)ex;
    if (threadIdx.x == 0) {
        unsigned long long total = s_warp[31];
        if ((long long)total > cap) {
            set_error(st, GS_ERR_CAPACITY, where);
            set_needed(st, (long long)total);
            *out_n = 0;
        } else {
            *out_n = (uint32_t)total;
        }
    }
}

// Pass B: the covering splats in id order: their depth keys, their tile
// rectangles and ids (one 16-byte entry each; depth and rectangle come from
// the 16 bytes of the record that hold both, one sector per splat) and their
// compacted index (the value the depth sort carries).  Each thread owns 8
// consecutive candidates of a 2048-candidate tile (one block scan per tile).
__global__ void __launch_bounds__(kSortThreads) compact_valid_kernel(
    const int32_t *__restrict__ tiles, const float4 *__restrict__ rec,
    const int32_t *__restrict__ view_start, int V, int k, long long cap_cand,
    const uint32_t *__restrict__ block_off, uint32_t *__restrict__ dkeys, uint4 *__restrict__ crec,
    uint32_t *__restrict__ cidx, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t C = (uint32_t)min((long long)__ldg(view_start + V) * k, cap_cand);
    uint32_t t0, t1;
    block_tiles(C, blockIdx.x, gridDim.x, &t0, &t1);
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_dk[kSortTile];
    __shared__ uint4 s_rec[kSortTile];
    const bool vec = (reinterpret_cast<uintptr_t>(tiles) & 15) == 0;
    uint32_t base = block_off[blockIdx.x];
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t i0 = t * kSortTile + threadIdx.x * kSortItems;
        int32_t tl[kSortItems];
        if (vec && i0 + kSortItems <= C) {
            const int4 u = __ldg(reinterpret_cast<const int4 *>(tiles + i0));
            const int4 w = __ldg(reinterpret_cast<const int4 *>(tiles + i0) + 1);
            tl[0] = u.x; tl[1] = u.y; tl[2] = u.z; tl[3] = u.w; tl[4] = w.x; tl[5] = w.y; tl[6] = w.z; tl[7] = w.w;
        } else {
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) tl[j] = i0 + j < C ? __ldg(tiles + i0 + j) : 0;
        }
        // record floats 8..11 (colour b, depth, rectangle) of the covering candidates, all loads
        // issued before the block scan
        float4 r[kSortItems];
        uint32_t n = 0;
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            r[j] = tl[j] > 0 ? __ldg(rec + 3 * (size_t)(i0 + j) + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
            n += tl[j] > 0;
        }
        uint32_t tot;
        uint32_t loc = scan256(n, s_warp, &tot);
        // staged in shared memory by tile-local position, then written out with consecutive
        // lanes on consecutive entries
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (tl[j] > 0) {
                if (idx_ok(st, (long long)loc, kSortTile, 31)) {
                    s_dk[loc] = __float_as_uint(r[j].y);
                    s_rec[loc] = make_uint4(__float_as_uint(r[j].z), __float_as_uint(r[j].w), i0 + j, 0u);
                }
                ++loc;
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tot; i += kSortThreads) {
            const uint32_t o = base + i;
            if (!idx_ok(st, (long long)o, C, 31)) break;
            dkeys[o] = s_dk[i];
            crec[o] = s_rec[i];
            cidx[o] = o;
        }
        __syncthreads();   // the stage is rewritten by the next tile
        base += tot;
    }
}

// Tile count of a packed rectangle (x0 | x1 << 16, y0 | y1 << 16).
__device__ __forceinline__ uint32_t rect_area(uint2 r)
{
    const int w = (int)(r.x >> 16) - (int)(r.x & 0xffffu), h = (int)(r.y >> 16) - (int)(r.y & 0xffffu);
    return w > 0 && h > 0 ? (uint32_t)(w * h) : 0u;
}

// Pairs: the covering splats' ids and tile rectangles gathered into depth
// order (from the compacted entries, by the compacted index the depth sort
// carried), read in order by the offsets and the emission, and per-block
// sums of their tile counts.  A covering splat with
// an empty rectangle is an inconsistent input (its tile count says
// otherwise).
__global__ void __launch_bounds__(kSortThreads) count_pairs_kernel(
    const uint32_t *__restrict__ cidx_s, const uint32_t *__restrict__ n_ptr, const uint4 *__restrict__ crec,
    uint32_t *__restrict__ ids, uint2 *__restrict__ rect,
    uint32_t *__restrict__ block_sums, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t S = *n_ptr;
    uint32_t t0, t1;
    block_tiles(S, blockIdx.x, gridDim.x, &t0, &t1);
    unsigned long long n = 0;
    for (uint32_t b = t0 * kSortTile; b < min(S, t1 * kSortTile); b += kSortThreads * kSortItems) {
        uint32_t q[kSortItems];
        uint4 r[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {   // the compacted indices, then the gathers, loads issued together
            const uint32_t i = b + j * kSortThreads + threadIdx.x;
            q[j] = i < S ? cidx_s[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const bool in = b + j * kSortThreads + threadIdx.x < S && q[j] < S;
            r[j] = in ? crec[q[j]] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t i = b + j * kSortThreads + threadIdx.x;
            if (i < S && idx_ok(st, q[j], S, 34)) {
                const uint2 rr = make_uint2(r[j].x, r[j].y);
                const uint32_t c = rect_area(rr);
                if (c == 0) idx_ok(st, (long long)r[j].z, -1, 34);
                rect[i] = rr;
                ids[i] = r[j].z;
                n += c;
            }
        }
    }
    // the per-block total fits 32 bits when the whole total does (checked later)
    __shared__ uint32_t s_warp[32];
    uint32_t tot;
    scan256((uint32_t)n, s_warp, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

constexpr int kEmitPairs = 2048;   // pairs written per CTA and round

// Per-splat pair offsets in depth order: offs[i] = sum of the tile counts of
// splats 0..i-1 (block prefixes from scan_block_sums), 8 splats per thread
// (their rectangles in four 16-byte loads) and one block scan per 2048
// splats.  Every splat owns >= 1 pair, so each emission round r (pairs
// [2048 r, 2048 r + 2048)) starts inside exactly one splat's range [offs[i],
// offs[i] + count): that splat writes round_first[r].
__global__ void __launch_bounds__(kSortThreads) pair_offsets_kernel(
    const uint2 *__restrict__ rect, const uint32_t *__restrict__ n_ptr, const uint32_t *__restrict__ block_off,
    uint32_t *__restrict__ offs, uint32_t *__restrict__ round_first, long long max_rounds, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t S = *n_ptr;
    uint32_t t0, t1;
    block_tiles(S, blockIdx.x, gridDim.x, &t0, &t1);
    __shared__ uint32_t s_warp[32];
    uint32_t base = block_off[blockIdx.x];
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t i0 = t * kSortTile + threadIdx.x * kSortItems;
        uint32_t cnt[kSortItems];
        uint32_t n = 0;
        if (i0 + kSortItems <= S) {
            const uint4 *r4 = reinterpret_cast<const uint4 *>(rect + i0);
            uint4 u[kSortItems / 2];
#pragma unroll
            for (int j = 0; j < kSortItems / 2; ++j) u[j] = r4[j];
#pragma unroll
            for (int j = 0; j < kSortItems / 2; ++j) {
                cnt[2 * j] = rect_area(make_uint2(u[j].x, u[j].y));
                cnt[2 * j + 1] = rect_area(make_uint2(u[j].z, u[j].w));
            }
        } else {
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) cnt[j] = i0 + j < S ? rect_area(rect[i0 + j]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) n += cnt[j];
        uint32_t tot;
        uint32_t off = base + scan256(n, s_warp, &tot);
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (i0 + j < S) {
                offs[i0 + j] = off;
                const unsigned long long end = (unsigned long long)off + cnt[j];
                for (unsigned long long r = ((unsigned long long)off + kEmitPairs - 1) / kEmitPairs;
                     r * kEmitPairs < end; ++r)
                    if (idx_ok(st, (long long)r, max_rounds, 37)) round_first[r] = i0 + j;
                off += cnt[j];
            }
        }
        base += tot;
    }
}

// Exclusive max-scan over the 256 threads of a block.
__device__ __forceinline__ uint32_t scanmax256_excl(uint32_t x, uint32_t *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = max(v, y);
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) ex = 0;
    for (int w = 0; w < warp; ++w) ex = max(ex, s_warp[w]);
    __syncthreads();
    return ex;
}

// Load-balanced emission: CTA rounds write pairs [p0, p0 + 2048).  The splats
// owning them run from round_first[r] (the splat holding p0) to
// round_first[r + 1] (the one holding the next round's first pair; it owns a
// pair of this round unless it starts exactly there) -- at most 2048 splats,
// since every compacted splat owns >= 1 pair.  Every thread reads the two
// bounds itself, and those of the CTA's next round are loaded while the
// current round runs.  The staged splats keep their rectangle's first tile
// (the rectangles come in depth order from count_pairs_kernel, read beside
// the ids), width and the view's tile row length; each marks the round-local position of its first pair in s_own
// and a max-scan fills every pair's position with its owner.  Pair t of a
// splat is tile (t % w, t / w) of its rectangle, row-major.
__global__ void __launch_bounds__(kSortThreads) emit_pairs_kernel(
    const uint32_t *__restrict__ ids, const uint32_t *__restrict__ n_ptr, const uint32_t *__restrict__ np_ptr,
    const uint32_t *__restrict__ offs, const uint32_t *__restrict__ round_first, const uint2 *__restrict__ rect,
    const int32_t *__restrict__ view_start, int k, uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals,
    ViewTable vt, long long cap_cand, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    constexpr int kPer = kEmitPairs / kSortThreads;   // staged splats / pairs per thread and round
    const uint32_t S = *n_ptr, P = *np_ptr;
    const uint32_t nrounds = (P + kEmitPairs - 1) / kEmitPairs;
    __shared__ uint32_t s_off[kEmitPairs], s_t00[kEmitPairs], s_id[kEmitPairs];
    __shared__ __align__(16) uint32_t s_own[kEmitPairs];
    __shared__ uint16_t s_w[kEmitPairs], s_tx[kEmitPairs];
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x;
    uint4 *own4 = reinterpret_cast<uint4 *>(s_own);
    uint32_t na = 0, nc = 0;   // bounds of the CTA's next round
    auto bounds = [&](uint32_t r) {
        na = round_first[r];
        nc = r + 1 < nrounds ? round_first[r + 1] : S - 1;
    };
    if (blockIdx.x < nrounds) bounds(blockIdx.x);
    for (uint32_t r = blockIdx.x; r < nrounds; r += gridDim.x) {
        const uint32_t p0 = r * (uint32_t)kEmitPairs, p1 = min(P, p0 + (uint32_t)kEmitPairs);
        const uint32_t sa = na, sc = nc;
        if (r + gridDim.x < nrounds) bounds(r + gridDim.x);
        uint32_t ns = 0;
        if (sa < S && sc < S && sc >= sa && sc - sa <= (uint32_t)kEmitPairs)
            ns = min(sc - sa + 1, (uint32_t)kEmitPairs);   // 2049 only if the last starts at p1
        else if (tid == 0)
            idx_ok(st, (long long)sc - (long long)sa, -1, 39);
#pragma unroll
        for (int q = 0; q < kPer / 4; ++q) own4[kPer / 4 * tid + q] = make_uint4(0u, 0u, 0u, 0u);
        uint32_t idv[kPer], ov[kPer], oe[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const uint32_t j = tid + u * kSortThreads;
            const bool in = j < ns;
            idv[u] = in ? ids[sa + j] : 0u;
            ov[u] = in ? offs[sa + j] : 0u;
            oe[u] = in ? (sa + j + 1 < S ? offs[sa + j + 1] : P) : 0u;
        }
        uint2 rv[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {   // the splats' rectangles, in depth order beside the ids
            const uint32_t j = tid + u * kSortThreads;
            rv[u] = j < ns ? rect[sa + j] : make_uint2(0u, 0u);
        }
        __syncthreads();   // s_own cleared (the previous round's readers are done)
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const uint32_t j = tid + u * kSortThreads;
            if (j >= ns) continue;
            const uint32_t id = idv[u];
            const uint32_t o = ov[u];
            uint32_t t00 = 0, w = 1, tx = 1;
            if (idx_ok(st, id, cap_cand, 36)) {
                const uint32_t rx = rv[u].x, ry = rv[u].y;
                const int x0 = rx & 0xffff, x1 = rx >> 16, y0 = ry & 0xffff, y1 = ry >> 16;
                const int v = view_of_row(view_start, vt.V, (int)(id / (uint32_t)k));
                // the splat's tile count from its offsets (no second read of tiles_touched)
                const long long cnt = (long long)oe[u] - (long long)o;
                if ((long long)(x1 - x0) * (y1 - y0) != cnt || x1 > vt.TX[v] || y1 > vt.TY[v] || x1 <= x0)
                    idx_ok(st, (long long)id, -1, 36);
                w = (uint32_t)max(x1 - x0, 1);
                tx = (uint32_t)vt.TX[v];
                t00 = (uint32_t)vt.tile_base[v] + (uint32_t)(y0 * vt.TX[v] + x0);
            }
            s_off[j] = o;
            s_t00[j] = t00;
            s_w[j] = (uint16_t)w;
            s_tx[j] = (uint16_t)tx;
            s_id[j] = id;
            if (o >= p1) continue;                      // starts at the next round's first pair
            const uint32_t at = o > p0 ? o - p0 : 0u;   // the first staged splat starts at or before p0
            if (j > 0 && o < p0) idx_ok(st, (long long)o, -1, 39);   // only the first may start before p0
            s_own[at] = j;
        }
        __syncthreads();
        {   // fill forward: thread t owns positions kPer t .. kPer t + kPer - 1
            uint32_t v[kPer];
#pragma unroll
            for (int q = 0; q < kPer / 4; ++q) {
                const uint4 x = own4[kPer / 4 * tid + q];
                v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
            }
            uint32_t m = 0;
#pragma unroll
            for (int u = 0; u < kPer; ++u) { m = max(m, v[u]); v[u] = m; }
            const uint32_t pre = scanmax256_excl(m, s_warp);
#pragma unroll
            for (int u = 0; u < kPer; ++u) v[u] = max(v[u], pre);
#pragma unroll
            for (int q = 0; q < kPer / 4; ++q)
                own4[kPer / 4 * tid + q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        __syncthreads();
        for (uint32_t i = tid; ns > 0 && p0 + i < p1; i += kSortThreads) {
            const uint32_t p = p0 + i, a = s_own[i];
            const uint32_t t = p - s_off[a], w = s_w[a];
            const uint32_t yy = t / w, xx = t - yy * w;
            tkeys[p] = s_t00[a] + yy * (uint32_t)s_tx[a] + xx;
            tvals[p] = s_id[a];
        }
        __syncthreads();
    }
}

// Tiles no pair touched keep the all-ones fill: empty range (0, 0); the
// others hold the complement of their end.
__global__ void __launch_bounds__(256) finish_ranges(uint32_t *__restrict__ ranges, int total_tiles,
                                                     const gs_status *st)
{
    if (has_error(st)) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        const uint2 r = reinterpret_cast<const uint2 *>(ranges)[t];
        reinterpret_cast<uint2 *>(ranges)[t] = r.x == 0xffffffffu ? make_uint2(0u, 0u) : make_uint2(r.x, ~r.y);
    }
}

__global__ void __launch_bounds__(256) keys_kernel(const uint32_t *__restrict__ tkeys,
                                                   const uint32_t *__restrict__ vals,
                                                   const uint32_t *__restrict__ n_ptr,
                                                   const float4 *__restrict__ rec,
                                                   unsigned long long *__restrict__ keys, const gs_status *st)
{
    if (has_error(st)) return;
    const uint32_t P = *n_ptr;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const uint32_t d = __float_as_uint(__ldg(&rec[3 * (size_t)vals[i] + 2]).y);
        keys[i] = ((unsigned long long)tkeys[i] << 32) | d;
    }
}

// ------------------------------------------------------------- host launch
struct SortLayout {
    size_t ids_a, ids_b, dk_a, dk_b, crec, offs, rect, rfirst, tk_a, tk_b, tv_b, hist, totals, sums, counts,
        total;
    long long max_rounds;
    int nb;
};

// CTAs of the sort and scan kernels: 4 per SM unless tuned (gs_set_tuning), at most 1024.
static int sort_blocks()
{
    const int per_sm = tuning().sort_ctas_per_sm > 0 ? tuning().sort_ctas_per_sm : 4;
    return std::max(1, std::min(1024, sm_count() * per_sm));
}

static SortLayout layout(long long cap_cand, long long cap_pairs)
{
    SortLayout L;
    L.nb = sort_blocks();
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.ids_a = take(sizeof(uint32_t) * std::max<long long>(cap_cand, 1));
    L.ids_b = take(sizeof(uint32_t) * std::max<long long>(cap_cand, 1));
    L.dk_a = take(sizeof(uint32_t) * std::max<long long>(cap_cand, 1));
    L.dk_b = take(sizeof(uint32_t) * std::max<long long>(cap_cand, 1));
    L.crec = take(sizeof(uint4) * std::max<long long>(cap_cand, 1));
    L.offs = take(sizeof(uint32_t) * std::max<long long>(cap_cand, 1));
    L.rect = take(sizeof(uint2) * std::max<long long>(cap_cand, 1));
    L.max_rounds = std::max<long long>(cap_pairs, 0) / kEmitPairs + 2;
    L.rfirst = take(sizeof(uint32_t) * (size_t)L.max_rounds);
    L.tk_a = take(sizeof(uint32_t) * std::max<long long>(cap_pairs, 1));
    L.tk_b = take(sizeof(uint32_t) * std::max<long long>(cap_pairs, 1));
    L.tv_b = take(sizeof(uint32_t) * std::max<long long>(cap_pairs, 1));
    L.hist = take(sizeof(uint32_t) * 256 * 1024);
    L.totals = take(sizeof(uint32_t) * 256);
    L.sums = take(sizeof(uint32_t) * 1024);
    L.counts = take(sizeof(uint32_t) * 4);
    L.total = o;
    return L;
}

size_t bin_sort_workspace_bytes(const ViewTable &vt, long long cap_cand, long long cap_pairs)
{
    (void)vt;
    return layout(cap_cand, cap_pairs).total;
}

// LSD radix sort of (key, value) over the low `bits` bits, 8 per pass.  The
// top digit is ranked by match_any (few distinct values in depth and tile
// keys); with `ranges`, the last pass also records the tile ranges.
static void radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const uint32_t *n_ptr,
                       int bits, uint32_t *hist, uint32_t *totals, int nb, gs_status *st, cudaStream_t s,
                       uint32_t **k_out, uint32_t **v_out, uint32_t *ranges = nullptr, int n_ranges = 0)
{
    for (int shift = 0; shift < bits; shift += 8) {
        radix_upsweep<<<nb, kSortThreads, 0, s>>>(k0, n_ptr, shift, hist, st);
        radix_scan_rows<<<256, 1024, 0, s>>>(hist, nb, totals, st);
        const bool top = shift + 8 >= bits;
        if (top && ranges)
            radix_downsweep<true, true><<<nb, kSortThreads, 0, s>>>(k0, v0, k1, v1, n_ptr, shift, hist, totals,
                                                                    ranges, n_ranges, st);
        else if (top)
            radix_downsweep<true, false><<<nb, kSortThreads, 0, s>>>(k0, v0, k1, v1, n_ptr, shift, hist, totals,
                                                                     nullptr, 0, st);
        else
            radix_downsweep<false, false><<<nb, kSortThreads, 0, s>>>(k0, v0, k1, v1, n_ptr, shift, hist, totals,
                                                                      nullptr, 0, st);
        std::swap(k0, k1);
        std::swap(v0, v1);
        count_launches(3);
    }
    *k_out = k0;
    *v_out = v0;
}

int launch_bin_sort(const gs_splats *sp, int k, const int32_t *view_start, long long cap_rows,
                    const ViewTable &vt, gs_bins *bins, void *ws, size_t ws_bytes, gs_status *st,
                    cudaStream_t s)
{
    const long long cap_cand = cap_rows * k;
    const SortLayout L = layout(cap_cand, bins->cap_pairs);
    if (ws_bytes < L.total) return GS_ERR_INVALID_ARG;
    char *w = reinterpret_cast<char *>(ws);
    uint32_t *ids_a = (uint32_t *)(w + L.ids_a), *ids_b = (uint32_t *)(w + L.ids_b);
    uint32_t *dk_a = (uint32_t *)(w + L.dk_a), *dk_b = (uint32_t *)(w + L.dk_b);
    uint32_t *tk_a = (uint32_t *)(w + L.tk_a), *tk_b = (uint32_t *)(w + L.tk_b);
    uint32_t *tv_b = (uint32_t *)(w + L.tv_b), *offs = (uint32_t *)(w + L.offs);
    uint32_t *rfirst = (uint32_t *)(w + L.rfirst);
    uint2 *rect = (uint2 *)(w + L.rect);
    uint4 *crec = (uint4 *)(w + L.crec);
    uint32_t *hist = (uint32_t *)(w + L.hist), *totals = (uint32_t *)(w + L.totals);
    uint32_t *sums = (uint32_t *)(w + L.sums), *counts = (uint32_t *)(w + L.counts);
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    const int nb = L.nb;
    uint32_t *n_splats = counts, *n_pairs = bins->n_pairs;

    // 1. compact covering splats
    count_valid_kernel<<<nb, kSortThreads, 0, s>>>(sp->tiles, view_start, vt.V, k, cap_cand, sums, st);
    scan_block_sums<<<1, 1024, 0, s>>>(sums, nb, n_splats, cap_cand, st, 3);
    compact_valid_kernel<<<nb, kSortThreads, 0, s>>>(sp->tiles, rec, view_start, vt.V, k, cap_cand, sums, dk_a, crec,
                                                     ids_a, st);
    count_launches(3);
    // 2. depth sort (32 bits) of the compacted indices
    uint32_t *dk_s, *ci_s;
    radix_sort(dk_a, ids_a, dk_b, ids_b, n_splats, 32, hist, totals, nb, st, s, &dk_s, &ci_s);
    // 3. pair emission in depth order (ids and rectangles gathered into it first)
    uint32_t *ids_s = ci_s == ids_a ? ids_b : ids_a;
    count_pairs_kernel<<<nb, kSortThreads, 0, s>>>(ci_s, n_splats, crec, ids_s, rect, sums, st);
    scan_block_sums<<<1, 1024, 0, s>>>(sums, nb, n_pairs, bins->cap_pairs, st, 3);
    int tile_bits = 1;
    while ((1ll << tile_bits) < (long long)vt.total_tiles) ++tile_bits;
    const int passes = (tile_bits + 7) / 8;
    // choose the emission buffers so that the last pass lands in bins->vals
    uint32_t *ek = tk_a, *ev = (passes % 2 == 0) ? bins->vals : tv_b;
    uint32_t *ok = tk_b, *ov = (passes % 2 == 0) ? tv_b : bins->vals;
    pair_offsets_kernel<<<nb, kSortThreads, 0, s>>>(rect, n_splats, sums, offs, rfirst, L.max_rounds, st);
    const int emit_per_sm = tuning().emit_ctas_per_sm > 0 ? std::min(tuning().emit_ctas_per_sm, 8) : 4;
    emit_pairs_kernel<<<sm_count() * emit_per_sm, kSortThreads, 0, s>>>(ids_s, n_splats, n_pairs, offs, rfirst, rect,
                                                              view_start, k, ek, ev, vt, cap_cand, st);
    count_launches(4);
    // 4. stable sort on the tile id
    // 5. tile ranges, recorded by the last pass (+ optional 64-bit keys)
    uint32_t *tk_s, *tv_s;
    cudaMemsetAsync(bins->ranges, 0xff, sizeof(uint32_t) * 2 * (size_t)vt.total_tiles, s);
    radix_sort(ek, ev, ok, ov, n_pairs, tile_bits, hist, totals, nb, st, s, &tk_s, &tv_s, bins->ranges,
               (int)vt.total_tiles);
    const int g = sm_count() * 8;
    finish_ranges<<<(int)std::min<long long>(g, (vt.total_tiles + 255) / 256), 256, 0, s>>>(bins->ranges,
                                                                                       (int)vt.total_tiles, st);
    count_launches(1);
    if (bins->keys) {
        keys_kernel<<<g, 256, 0, s>>>(tk_s, tv_s, n_pairs, rec, reinterpret_cast<unsigned long long *>(bins->keys), st);
        count_launches(1);
    }
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// ------------------------------------------------------------ voxelisation
// Eq. 4: V = unique(round(P / eps)) * eps, for the map's incremental growth.
// Each point's voxel index (i, j, l) = rint(p / eps) (one correctly rounded
// single-precision division, ties to even) is packed into the 64-bit key
// ((i + 2^20) << 42) | ((j + 2^20) << 21) | (l + 2^20); the keys are sorted
// with the radix sort above (low word, then high word, stable), and the first
// key of every run that is not among the caller's existing keys is written in
// ascending order with its centre index * eps.
constexpr int kVoxBias = 1 << 20;

__global__ void __launch_bounds__(256) voxel_keys_kernel(const float *__restrict__ pts, uint32_t P, float eps,
                                                         uint32_t *__restrict__ lo, uint32_t *__restrict__ hi,
                                                         uint32_t *__restrict__ lo_sort, uint32_t *__restrict__ idx,
                                                         uint32_t *__restrict__ count, gs_status *st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = P;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        unsigned long long key = 0;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float r = rintf(__fdiv_rn(__ldg(pts + 3 * (size_t)i + a), eps));
            ok = ok && r > -(float)kVoxBias && r < (float)kVoxBias;
            key = (key << 21) | (unsigned long long)(ok ? (int)r + kVoxBias : 0);
        }
        if (!ok) set_error(st, GS_ERR_INVALID_ARG, 80);
        lo[i] = (uint32_t)key;
        hi[i] = (uint32_t)(key >> 32);
        lo_sort[i] = (uint32_t)key;
        idx[i] = i;
    }
}

__global__ void __launch_bounds__(256) gather_u32_kernel(const uint32_t *__restrict__ src,
                                                         const uint32_t *__restrict__ idx,
                                                         uint32_t *__restrict__ dst, const uint32_t *__restrict__ n_ptr,
                                                         const gs_status *st)
{
    if (has_error(st)) return;
    const uint32_t n = *n_ptr;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t j = idx[i];
        dst[i] = idx_ok(st, j, n, 81) ? src[j] : 0u;
    }
}

// Whether sorted position i starts a run whose key is not in `existing`.
__device__ __forceinline__ bool voxel_is_new(uint32_t i, const uint32_t *__restrict__ hi,
                                             const uint32_t *__restrict__ lo,
                                             const unsigned long long *__restrict__ existing, long long n_ex,
                                             unsigned long long *key)
{
    const unsigned long long k = ((unsigned long long)hi[i] << 32) | lo[i];
    *key = k;
    if (i > 0 && k == (((unsigned long long)hi[i - 1] << 32) | lo[i - 1])) return false;
    long long a = 0, b = n_ex;   // first position with existing >= k
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (existing[m] < k) a = m + 1; else b = m;
    }
    return !(a < n_ex && existing[a] == k);
}

__global__ void __launch_bounds__(kSortThreads) voxel_count_kernel(const uint32_t *__restrict__ hi,
                                                                   const uint32_t *__restrict__ lo,
                                                                   const uint32_t *__restrict__ n_ptr,
                                                                   const unsigned long long *__restrict__ existing,
                                                                   long long n_ex, uint32_t *__restrict__ block_sums,
                                                                   const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t n = *n_ptr;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, &t0, &t1);
    uint32_t c = 0;
    unsigned long long k;
    for (uint32_t i = t0 * kSortTile + threadIdx.x; i < min(n, t1 * kSortTile); i += kSortThreads)
        c += voxel_is_new(i, hi, lo, existing, n_ex, &k);
    __shared__ uint32_t s_warp[32];
    uint32_t tot;
    scan256(c, s_warp, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kSortThreads) voxel_write_kernel(const uint32_t *__restrict__ hi,
                                                                   const uint32_t *__restrict__ lo,
                                                                   const uint32_t *__restrict__ n_ptr,
                                                                   const unsigned long long *__restrict__ existing,
                                                                   long long n_ex,
                                                                   const uint32_t *__restrict__ block_off, float eps,
                                                                   unsigned long long *__restrict__ keys_out,
                                                                   float *__restrict__ centers_out, long long cap,
                                                                   const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const uint32_t n = *n_ptr;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, &t0, &t1);
    __shared__ uint32_t s_warp[32];
    uint32_t base = block_off[blockIdx.x];
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t i0 = t * kSortTile + threadIdx.x * kSortItems;
        bool nw[kSortItems];
        unsigned long long key[kSortItems];
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            nw[j] = i0 + j < n && voxel_is_new(i0 + j, hi, lo, existing, n_ex, &key[j]);
            c += nw[j];
        }
        uint32_t tot;
        uint32_t off = base + scan256(c, s_warp, &tot);
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (!nw[j]) continue;
            if (idx_ok(st, (long long)off, cap, 82)) {
                keys_out[off] = key[j];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int v = (int)((key[j] >> (42 - 21 * a)) & 0x1FFFFFull) - kVoxBias;
                    centers_out[3 * (size_t)off + a] = __fmul_rn((float)v, eps);
                }
            }
            ++off;
        }
        base += tot;
    }
}

struct VoxLayout {
    size_t lo, hi, ka, kb, va, vb, hist, totals, sums, counts, total;
    int nb;
};

static VoxLayout vox_layout(long long P)
{
    VoxLayout L;
    L.nb = sort_blocks();
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    const size_t n = sizeof(uint32_t) * (size_t)std::max<long long>(P, 1);
    L.lo = take(n); L.hi = take(n); L.ka = take(n); L.kb = take(n); L.va = take(n); L.vb = take(n);
    L.hist = take(sizeof(uint32_t) * 256 * 1024);
    L.totals = take(sizeof(uint32_t) * 256);
    L.sums = take(sizeof(uint32_t) * 1024);
    L.counts = take(sizeof(uint32_t) * 4);
    L.total = o;
    return L;
}

size_t voxelize_workspace_bytes(long long P) { return vox_layout(P).total; }

int launch_voxelize(const float *pts, long long P, float eps, const unsigned long long *existing, long long n_ex,
                    unsigned long long *keys_out, float *centers_out, long long cap, uint32_t *n_out, void *ws,
                    gs_status *st, cudaStream_t s)
{
    const VoxLayout L = vox_layout(P);
    char *w = reinterpret_cast<char *>(ws);
    uint32_t *lo = (uint32_t *)(w + L.lo), *hi = (uint32_t *)(w + L.hi);
    uint32_t *ka = (uint32_t *)(w + L.ka), *kb = (uint32_t *)(w + L.kb);
    uint32_t *va = (uint32_t *)(w + L.va), *vb = (uint32_t *)(w + L.vb);
    uint32_t *hist = (uint32_t *)(w + L.hist), *totals = (uint32_t *)(w + L.totals);
    uint32_t *sums = (uint32_t *)(w + L.sums), *count = (uint32_t *)(w + L.counts);
    const int g = (int)std::max<long long>(1, std::min<long long>((P + 255) / 256, (long long)sm_count() * 8));
    voxel_keys_kernel<<<g, 256, 0, s>>>(pts, (uint32_t)P, eps, lo, hi, ka, va, count, st);
    count_launches(1);
    uint32_t *k1, *v1;   // sorted by the low word
    radix_sort(ka, va, kb, vb, count, 32, hist, totals, L.nb, st, s, &k1, &v1);
    uint32_t *kf = (k1 == ka) ? kb : ka, *vf = (v1 == va) ? vb : va;   // the free pair
    gather_u32_kernel<<<g, 256, 0, s>>>(hi, v1, kf, count, st);
    count_launches(1);
    uint32_t *k2, *v2;   // then stably by the high word (31 bits)
    radix_sort(kf, v1, k1, vf, count, 31, hist, totals, L.nb, st, s, &k2, &v2);
    uint32_t *lo2 = (k2 == kf) ? k1 : kf;   // the key buffer not holding the result
    gather_u32_kernel<<<g, 256, 0, s>>>(lo, v2, lo2, count, st);
    count_launches(1);
    voxel_count_kernel<<<L.nb, kSortThreads, 0, s>>>(k2, lo2, count, existing, n_ex, sums, st);
    scan_block_sums<<<1, 1024, 0, s>>>(sums, L.nb, n_out, cap, st, 8);
    voxel_write_kernel<<<L.nb, kSortThreads, 0, s>>>(k2, lo2, count, existing, n_ex, sums, eps, keys_out, centers_out,
                                                     cap, st);
    count_launches(3);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
