// Tile binning and depth sort (Section 3: "sorts points according to
// view-dependent depth" before alpha compositing).
//
// Order produced: instances (Gaussian i, tile t) sorted by (t, depth bits of
// i, i).  Design: a stable LSD radix sort of the N Gaussians on their float32
// depth bits (32 bits), emission of each Gaussian's instances in that order,
// then a stable LSD radix sort of the M instances on the tile id only
// (ceil(log2 T) bits).  Because the second sort is stable and its input is in
// (depth, i) order, the result equals one stable sort of the 64-bit keys
// (t << 32 | depth bits) emitted in Gaussian order, at a fraction of the
// passes over the M instances.
#include "common.cuh"

namespace sgs {

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (three phases: block sums, scan of the sums,
// block-local scans with carried offset).
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SCAN_MAX_BLOCKS = 1024;

static int scan_blocks(int64_t n_max) {
    int64_t b = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    if (b < 1) b = 1;
    if (b > SCAN_MAX_BLOCKS) b = SCAN_MAX_BLOCKS;
    return (int)b;
}

size_t scan_tmp_bytes(int64_t n_max) {
    return sizeof(uint32_t) * (size_t)(scan_blocks(n_max) + 1) + 256;
}

__device__ __forceinline__ int64_t read_n(const int32_t* d_n, int64_t n_host, int64_t cap) {
    int64_t n = d_n ? (int64_t)(*d_n) : n_host;
    if (n < 0) n = 0;
    return n < cap ? n : cap;
}

// Inclusive scan of one value per thread across a block of SCAN_THREADS.
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t add = warp > 0 ? s_warp[warp - 1] : 0u;
    __syncthreads();
    return v + add;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                                   const int32_t* d_n, int64_t n_max,
                                                                   uint32_t* __restrict__ partial) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[32];
    int64_t n = read_n(d_n, n_max, n_max);
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    int64_t start = (int64_t)blockIdx.x * chunk, end = min(n, start + chunk);
    uint32_t sum = 0;
    for (int64_t i = start + threadIdx.x; i < end; i += blockDim.x) sum += in[i];
    sum = block_inclusive_scan(sum, s_warp);
    if (threadIdx.x == blockDim.x - 1) partial[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_partials_kernel(uint32_t* __restrict__ partial,
                                                                     int nb, uint32_t* __restrict__ d_total) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[32];
    uint32_t v = threadIdx.x < nb ? partial[threadIdx.x] : 0u;
    uint32_t inc = block_inclusive_scan(v, s_warp);
    if (threadIdx.x < nb) partial[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1 && d_total) *d_total = inc;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_downsweep_kernel(
    const uint32_t* __restrict__ in, uint32_t* __restrict__ out, const int32_t* d_n, int64_t n_max,
    const uint32_t* __restrict__ partial, int64_t fixed_chunk) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    int64_t n = read_n(d_n, n_max, n_max);
    int64_t chunk = fixed_chunk > 0 ? fixed_chunk : (n + gridDim.x - 1) / gridDim.x;
    int64_t start = (int64_t)blockIdx.x * chunk, end = min(n, start + chunk);
    if (threadIdx.x == 0) s_carry = partial[blockIdx.x];
    __syncthreads();
    for (int64_t base = start; base < end; base += SCAN_TILE) {
        int64_t i0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = (i0 + k < end) ? in[i0 + k] : 0u;
            sum += v[k];
        }
        uint32_t inc = block_inclusive_scan(sum, s_warp);
        uint32_t run = s_carry + inc - sum;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (i0 + k < end) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += inc;
        __syncthreads();
    }
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t* d_total, int64_t n_max,
                                  const int32_t* d_n, void* tmp, cudaStream_t stream) {
    int nb = scan_blocks(n_max);
    uint32_t* partial = reinterpret_cast<uint32_t*>(tmp);
    (void)launch_pdl(scan_reduce_kernel, dim3(nb), dim3(SCAN_THREADS), 0, stream, in, d_n, n_max, partial);
    note_launch();
    (void)launch_pdl(scan_partials_kernel, dim3(1), dim3(SCAN_THREADS), 0, stream, partial, nb, d_total);
    note_launch();
    (void)launch_pdl(scan_downsweep_kernel, dim3(nb), dim3(SCAN_THREADS), 0, stream, in, out, d_n, n_max, partial,
                     (int64_t)0);
    note_launch();
    return cudaGetLastError();
}

// Chunk sums from the producer's 256-value block sums: chunk c covers blocks
// [c per, (c + 1) per); exclusive prefixes over the chunks and the total.
__global__ void __launch_bounds__(SCAN_THREADS) scan_partials_counted_kernel(
    const uint32_t* __restrict__ bcount, int nbe, int per, uint32_t* __restrict__ partial, int nb,
    uint32_t* __restrict__ d_total) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[32];
    uint32_t v = 0u;
    if ((int)threadIdx.x < nb) {
        const int b0 = (int)threadIdx.x * per, b1 = min(nbe, b0 + per);
        for (int b = b0; b < b1; ++b) v += bcount[b];
    }
    const uint32_t inc = block_inclusive_scan(v, s_warp);
    if ((int)threadIdx.x < nb) partial[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1 && d_total) *d_total = inc;
}

cudaError_t launch_exclusive_scan_counted(const uint32_t* in, uint32_t* out, uint32_t* d_total, int64_t n,
                                          const uint32_t* bcount, void* tmp, cudaStream_t stream) {
    const int64_t nbe = (n + 255) / 256;
    const int nb_max = scan_blocks(n);          // chunks: at most the plain scan's, so tmp suffices
    int64_t per = (nbe + nb_max - 1) / nb_max;
    if (per < SCAN_TILE / 256) per = SCAN_TILE / 256;
    const int nb = (int)((nbe + per - 1) / per);
    uint32_t* partial = reinterpret_cast<uint32_t*>(tmp);
    (void)launch_pdl(scan_partials_counted_kernel, dim3(1), dim3(SCAN_THREADS), 0, stream, bcount, (int)nbe,
                     (int)per, partial, nb, d_total);
    note_launch();
    (void)launch_pdl(scan_downsweep_kernel, dim3(nb), dim3(SCAN_THREADS), 0, stream, in, out, nullptr, n, partial,
                     per * 256);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable LSD radix passes (reduce, scan, scatter) with chunked blocks.
//
// A pass over n items runs G blocks (G <= SORT_G_MAX, fixed on the host); block
// b owns the contiguous chunk [b C, min(n, (b + 1) C)), C = ceil(n / G), and
// walks it in tiles of RS_TILE items.  hist[d][b] = count of digit d in chunk
// b; one scan kernel turns each digit's row into exclusive prefixes over the
// blocks and writes the digit totals; the scatter ranks each tile's items per
// digit in item order (warp ballots + a cross-warp prefix) and writes item k of
// digit d to  base[d] + prefix[d][b] + rank,  so the pass is stable.  Each
// pass's per-block counts come from a counting kernel over its input (the
// first tile pass's from the emission, which writes that input).
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_MAX_BITS = 8;
constexpr int RS_RADIX_MAX = 1 << RS_MAX_BITS;
constexpr int SORT_G_MAX = 1024;             // blocks of one pass (= threads of the scan kernel)
constexpr int kSortPdlMaxRows = 4 << 20;     // dependent launches for sorts of at most this many rows
constexpr int DEPTH_PASSES = 4;              // 32 depth bits
constexpr int TILE_PASSES_MAX = 4;           // tile ids < 2^31
constexpr int EMIT_THREADS = 256;
constexpr int EMIT_SUB = 1024;               // rows staged per emission round
constexpr int EMIT_G_MAX = 4096;             // emission blocks (4 per thread of the offsets scan)
constexpr int EMIT_ROWS_PER_BLOCK = 256;     // target rows per emission block (of all rows)
constexpr int EMIT_SPAN = 8;                 // next-pass blocks gathered in shared memory per round
constexpr int EMIT_STAGE = 2048;             // instances staged in shared memory per write-out
constexpr int EMIT_DIRECT_MAX = 4 * EMIT_THREADS;   // rounds up to this many instances write directly
static_assert(EMIT_THREADS == RS_RADIX_MAX, "emit sums one depth digit total per thread");
static_assert(EMIT_SUB % EMIT_THREADS == 0, "emit rows per thread");

static int sort_blocks(int64_t n_max, int64_t per_block) {
    int64_t g = (n_max + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > SORT_G_MAX) g = SORT_G_MAX;
    return (int)g;
}

__device__ __forceinline__ int64_t chunk_of(int64_t n, int G) { return (n + G - 1) / G; }

struct PassDesc {
    int shift, bits;
    uint32_t* hist;          // [1 << bits][G]: counts, then (after the scan) exclusive prefixes
    uint32_t* tot;           // [1 << bits] digit totals (written by the scan)
    int G;
};

struct NextHist {            // per-block histogram of the following pass (bits = 0: none)
    int shift, bits;
    uint32_t* hist;          // [1 << bits][G]
    int G;
};

// Exclusive scan of one digit's per-block counts (one block per digit).
__global__ void __launch_bounds__(SORT_G_MAX) pass_scan_kernel(uint32_t* __restrict__ hist, int G,
                                                               uint32_t* __restrict__ tot) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[32];
    uint32_t* h = hist + (size_t)blockIdx.x * G;
    const uint32_t v = threadIdx.x < G ? h[threadIdx.x] : 0u;
    const uint32_t inc = block_inclusive_scan(v, s_warp);
    if (threadIdx.x < G) h[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1) tot[blockIdx.x] = inc;
}

// Lanes with the same digit as this lane (an invalid item has its own class):
// bits ballots instead of a match instruction.
__device__ __forceinline__ unsigned digit_peers(uint32_t dig, bool valid, int bits) {
    unsigned m = __ballot_sync(0xffffffffu, valid);
    m = valid ? m : ~m;
    for (int b = 0; b < bits; ++b) {
        const bool one = (dig >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, one);
        m &= one ? bal : ~bal;
    }
    return m;
}

// Counts of the first depth pass per block over the projection rows; only rows
// with tiles_touched > 0 are items (their float32 depth bits are the key: depth
// > near_z > 0, so the bits order like the value).
__global__ void __launch_bounds__(RS_THREADS) depth_hist_first_kernel(const float* __restrict__ depth,
                                                                      const uint32_t* __restrict__ tiles_touched,
                                                                      int64_t n_rows, PassDesc ps) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_h[RS_RADIX_MAX];
    for (int k = threadIdx.x; k < RS_RADIX_MAX; k += RS_THREADS) s_h[k] = 0u;
    __syncthreads();
    const int64_t C = chunk_of(n_rows, ps.G);
    const int64_t lo = (int64_t)blockIdx.x * C, hi = min(n_rows, lo + C);
    const int lane = threadIdx.x & 31;
    const uint32_t mask = (1u << ps.bits) - 1u;
    // RS_ITEMS rows per thread loaded before any is counted (one memory
    // round trip per RS_TILE rows instead of one per RS_THREADS)
    for (int64_t base = lo; base < hi; base += RS_TILE) {
        uint32_t t[RS_ITEMS], b[RS_ITEMS];
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const int64_t i = base + it * RS_THREADS + threadIdx.x;
            t[it] = i < hi ? tiles_touched[i] : 0u;
            b[it] = i < hi ? __float_as_uint(depth[i]) : 0u;
        }
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            if (base + it * RS_THREADS >= hi) break;    // block-uniform
            const bool valid = t[it] != 0u;
            const uint32_t d = valid ? ((b[it] >> ps.shift) & mask) : 0u;
            const unsigned peers = digit_peers(d, valid, ps.bits);
            if (valid && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << ps.bits); d += RS_THREADS) ps.hist[(size_t)d * ps.G + blockIdx.x] = s_h[d];
}

// Per-block digit counts of a pass whose items are keys[0, total of the
// previous pass) (the previous pass's output).
__global__ void __launch_bounds__(RS_THREADS) pass_hist_kernel(const uint32_t* __restrict__ keys,
                                                               const uint32_t* __restrict__ prev_tot, int prev_radix,
                                                               PassDesc ps) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_h[RS_RADIX_MAX];
    __shared__ uint32_t s_n;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_n = 0u;
    for (int k = threadIdx.x; k < RS_RADIX_MAX; k += RS_THREADS) s_h[k] = 0u;
    __syncthreads();
    {
        uint32_t c = threadIdx.x < prev_radix ? prev_tot[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) atomicAdd(&s_n, c);
    }
    __syncthreads();
    const int64_t n = s_n;
    const int64_t C = chunk_of(n, ps.G);
    const int64_t lo = (int64_t)blockIdx.x * C, hi = min(n, lo + C);
    const uint32_t mask = (1u << ps.bits) - 1u;
    for (int64_t base = lo; base < hi; base += RS_TILE) {
        uint32_t k[RS_ITEMS];
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const int64_t i = base + it * RS_THREADS + threadIdx.x;
            k[it] = i < hi ? keys[i] : 0u;
        }
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            if (base + it * RS_THREADS >= hi) break;    // block-uniform
            const bool valid = base + it * RS_THREADS + threadIdx.x < hi;
            const uint32_t d = valid ? ((k[it] >> ps.shift) & mask) : 0u;
            const unsigned peers = digit_peers(d, valid, ps.bits);
            if (valid && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << ps.bits); d += RS_THREADS) ps.hist[(size_t)d * ps.G + blockIdx.x] = s_h[d];
}

// One stable pass.  FIRST: items are the projection rows [0, n_rows) (rows
// that touch no tile are dropped), key = depth bits, value = row.  Otherwise
// items are (keys_in, vals_in)[0, total of the pass).  keys_out may be NULL.
// GATHER (last depth pass): also writes cnt_out[dest] = tiles_touched[value]
// and adds it to esum[dest chunk] (the emission's per-block instance counts).
template <bool FIRST, bool GATHER>
__global__ void __launch_bounds__(RS_THREADS) pass_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, const float* __restrict__ depth,
    const uint32_t* __restrict__ tiles_touched, int64_t n_rows, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, PassDesc ps, uint32_t* __restrict__ cnt_out,
    unsigned long long* __restrict__ esum, int G_emit) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_warp[RS_WARPS][RS_RADIX_MAX + 1];
    __shared__ uint32_t s_off[RS_RADIX_MAX];
    __shared__ uint32_t s_tot[RS_RADIX_MAX];
    __shared__ uint32_t s_lbase[RS_RADIX_MAX];
    __shared__ uint32_t s_key[RS_TILE];
    __shared__ uint32_t s_val[RS_TILE];
    __shared__ uint32_t s_scan[32];
    __shared__ uint32_t s_ntile;
    const int radix = 1 << ps.bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // digit bases: exclusive scan of the totals (radix <= RS_THREADS)
    const uint32_t tv = threadIdx.x < radix ? ps.tot[threadIdx.x] : 0u;
    const uint32_t tinc = block_inclusive_scan(tv, s_scan);
    if (threadIdx.x == RS_THREADS - 1) s_scan[31] = tinc;     // total (block_inclusive_scan ends synced)
    __syncthreads();
    const int64_t n_out = s_scan[31];
    const int64_t n_items = FIRST ? n_rows : n_out;
    const int64_t C = chunk_of(n_items, ps.G);
    const int64_t lo = (int64_t)blockIdx.x * C, hi = min(n_items, lo + C);
    if (threadIdx.x < radix) s_off[threadIdx.x] = (tinc - tv) + ps.hist[(size_t)threadIdx.x * ps.G + blockIdx.x];
    const uint32_t C_emit = GATHER ? (uint32_t)chunk_of(n_out, G_emit) : 1u;

    for (int64_t tile = lo; tile < hi; tile += RS_TILE) {
        for (int k = threadIdx.x; k < RS_WARPS * (RS_RADIX_MAX + 1); k += RS_THREADS) (&s_warp[0][0])[k] = 0u;
        __syncthreads();
        uint32_t key[RS_ITEMS], val[RS_ITEMS], dig[RS_ITEMS], rank[RS_ITEMS];
        bool ok[RS_ITEMS];
        // the tile's items split into 8 contiguous warp chunks (a multiple of
        // 32 each), so that a short tile spreads over all warps
        const int tile_n = (int)min((int64_t)RS_TILE, hi - tile);
        const int wchunk = (((tile_n + RS_WARPS - 1) / RS_WARPS) + 31) & ~31;
        const int iters = wchunk >> 5;
        const int64_t wbase = tile + (int64_t)warp * wchunk + lane;
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const int64_t idx = wbase + it * 32;
            bool valid = it < iters && idx < hi;
            if (FIRST) {
                valid = valid && tiles_touched[idx] != 0u;
                key[it] = valid ? __float_as_uint(depth[idx]) : 0u;
                val[it] = (uint32_t)idx;
            } else {
                key[it] = valid ? keys_in[idx] : 0u;
                val[it] = valid ? vals_in[idx] : 0u;
            }
            ok[it] = valid;
            dig[it] = (key[it] >> ps.shift) & mask;
        }
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            if (it >= iters) break;                     // block-uniform
            const unsigned peers = digit_peers(dig[it], ok[it], ps.bits);
            const unsigned lower = peers & ((1u << lane) - 1u);
            const uint32_t slot = ok[it] ? dig[it] : (uint32_t)radix;
            const uint32_t b = s_warp[warp][slot];
            rank[it] = b + (uint32_t)__popc(lower);
            __syncwarp();
            if (lower == 0u) s_warp[warp][slot] = b + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t dtot = 0;
        if (threadIdx.x < radix) {
            const int d = threadIdx.x;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = s_warp[w][d];
                s_warp[w][d] = dtot;
                dtot += c;
            }
            s_tot[d] = dtot;
        }
        // local sort of the tile by digit in shared memory, so that the
        // global writes below go out as runs of consecutive addresses
        const uint32_t linc = block_inclusive_scan(dtot, s_scan);   // (ends synced)
        if (threadIdx.x < radix) s_lbase[threadIdx.x] = linc - dtot;
        if (threadIdx.x == RS_THREADS - 1) s_ntile = linc;
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            if (!ok[it]) continue;
            const uint32_t lp = s_lbase[dig[it]] + s_warp[warp][dig[it]] + rank[it];
            s_key[lp] = key[it];
            s_val[lp] = val[it];
        }
        __syncthreads();
        const uint32_t ntile = s_ntile;
        for (uint32_t i0 = 0; i0 < ntile; i0 += RS_THREADS) {
            const uint32_t i = i0 + threadIdx.x;
            const bool okk = i < ntile;
            const uint32_t k = okk ? s_key[i] : 0u;
            const uint32_t vv = okk ? s_val[i] : 0u;
            const uint32_t d = (k >> ps.shift) & mask;
            const uint32_t dest = okk ? s_off[d] + (i - s_lbase[d]) : 0u;
            if (okk) {
                if (keys_out) keys_out[dest] = k;
                vals_out[dest] = vv;
            }
            if (GATHER) {
                // tile counts in depth order, summed per emission block; the
                // lanes of a warp usually share the block: one add per warp
                const uint32_t c = okk ? tiles_touched[vv] : 0u;
                if (okk) cnt_out[dest] = c;
                const uint32_t eb = okk ? dest / C_emit : 0xffffffffu;
                const uint32_t eb0 = __shfl_sync(0xffffffffu, eb, 0);
                if (__all_sync(0xffffffffu, eb == eb0 || !okk)) {
                    unsigned long long sum = c;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                    if (lane == 0 && sum) atomicAdd(esum + eb0, sum);
                } else if (okk && c) {
                    atomicAdd(esum + eb, (unsigned long long)c);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < radix) s_off[threadIdx.x] += s_tot[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan of the emission blocks' instance counts (one block of
// SORT_G_MAX threads, EMIT_G_MAX / SORT_G_MAX consecutive counts per thread);
// writes M.
__global__ void __launch_bounds__(SORT_G_MAX) emit_offsets_kernel(unsigned long long* __restrict__ esum, int G,
                                                                  int32_t* __restrict__ d_count) {
    pdl_wait_and_trigger();
    constexpr int PER = EMIT_G_MAX / SORT_G_MAX;
    __shared__ unsigned long long s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long v[PER], mine = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x * PER + q;
        v[q] = i < G ? esum[i] : 0ull;
        mine += v[q];
    }
    unsigned long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    const unsigned long long inc = x + (warp > 0 ? s_w[warp - 1] : 0ull);
    unsigned long long run = inc - mine;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x * PER + q;
        if (i < G) esum[i] = run;
        run += v[q];
    }
    if (threadIdx.x == blockDim.x - 1) *d_count = inc > 0x7fffffffull ? 0x7fffffff : (int32_t)inc;
}

// Emission of the (tile, row) instances in depth order, load-balanced: block b
// owns the depth-sorted rows of chunk b; per round of EMIT_SUB rows it scans
// their counts into shared memory and then spreads the round's instances over
// all threads (instance k -> its row by binary search, its tile from the
// offset inside the row's rect, row-major), so consecutive threads write
// consecutive positions.  At most `cap` instances are written; the first
// tile pass's per-block histogram is counted from the written positions.
template <bool STAGED>
__global__ void __launch_bounds__(EMIT_THREADS) emit_kernel(
    const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cnt, const short4* __restrict__ rect,
    const uint32_t* __restrict__ depth_tot, ViewsDev vd, int64_t cap, const unsigned long long* __restrict__ esum,
    int G_emit, const int32_t* __restrict__ d_count, uint32_t* __restrict__ inst_tile,
    uint32_t* __restrict__ inst_gid, NextHist nh) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_off[EMIT_SUB + 1];
    __shared__ uint32_t s_row[EMIT_SUB];
    __shared__ short4 s_rect[EMIT_SUB];
    __shared__ uint32_t s_warp[EMIT_THREADS / 32];
    __shared__ uint32_t s_nh[RS_RADIX_MAX][EMIT_SPAN];
    __shared__ uint32_t s_et[STAGED ? EMIT_STAGE : 1];   // a chunk's tile ids and rows, written out coalesced
    __shared__ uint32_t s_eg[STAGED ? EMIT_STAGE : 1];
    __shared__ uint32_t s_nvis;
    // per-view row bounds, tile offsets and tile-grid widths in shared memory:
    // the rows of one round come from different views, and indexing the kernel
    // parameters with a lane-dependent view serialises the constant loads
    __shared__ int s_rowoff[kMaxViews + 1];
    __shared__ uint32_t s_tileoff[kMaxViews];
    __shared__ int s_gx[kMaxViews];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_nvis = 0u;
    if (threadIdx.x <= vd.nv) s_rowoff[threadIdx.x] = (int)vd.row_off[threadIdx.x];
    if (threadIdx.x < vd.nv) {
        s_tileoff[threadIdx.x] = (uint32_t)vd.tile_off[threadIdx.x];
        s_gx[threadIdx.x] = vd.cam[threadIdx.x].gx;
    }
    __syncthreads();
    const int nv = vd.nv;
    auto view_of = [&](uint32_t row) {
        int v = 0;
        while (v + 1 < nv && (int)row >= s_rowoff[v + 1]) ++v;
        return v;
    };
    {
        uint32_t c = depth_tot[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) atomicAdd(&s_nvis, c);
    }
    __syncthreads();
    const int64_t n_vis = s_nvis;
    const int64_t C = chunk_of(n_vis, G_emit);
    const int64_t lo = (int64_t)blockIdx.x * C, hi = min(n_vis, lo + C);
    const int64_t M = *d_count;
    const int64_t n_written = M < cap ? M : cap;
    const uint32_t C_next = nh.bits > 0 ? (uint32_t)chunk_of(n_written, nh.G) : 1u;
    const uint32_t nmask = (1u << nh.bits) - 1u;
    int64_t base = (int64_t)esum[blockIdx.x];
    for (int64_t r0 = lo; r0 < hi; r0 += EMIT_SUB) {
        const int rows = (int)min((int64_t)EMIT_SUB, hi - r0);
        // counts of this round's rows: 4 consecutive rows per thread, block scan
        uint32_t c[EMIT_SUB / EMIT_THREADS];
        uint32_t mine = 0;
#pragma unroll
        for (int q = 0; q < EMIT_SUB / EMIT_THREADS; ++q) {
            const int j = threadIdx.x * (EMIT_SUB / EMIT_THREADS) + q;
            c[q] = j < rows ? cnt[r0 + j] : 0u;
            mine += c[q];
            if (j < rows) {
                const uint32_t g = perm[r0 + j];
                s_row[j] = g;
                s_rect[j] = rect[g];
            }
        }
        uint32_t x = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = 0;
            for (int w = 0; w < EMIT_THREADS / 32; ++w) {
                const uint32_t t = s_warp[w];
                s_warp[w] = run;
                run += t;
            }
            s_off[EMIT_SUB] = run;
        }
        __syncthreads();
        {
            uint32_t o = s_warp[warp] + x - mine;
#pragma unroll
            for (int q = 0; q < EMIT_SUB / EMIT_THREADS; ++q) {
                const int j = threadIdx.x * (EMIT_SUB / EMIT_THREADS) + q;
                if (j < rows) s_off[j] = o;
                o += c[q];
            }
        }
        const uint32_t total = s_off[EMIT_SUB];
        // the round's positions fall in next-pass blocks [nb0, nb0 + span);
        // with a small span their histogram is gathered in shared memory
        const int64_t last_pos = min(base + (int64_t)total, n_written) - 1;
        const uint32_t nb0 = base < n_written ? (uint32_t)base / C_next : 0u;
        const int span = last_pos >= base ? (int)((uint32_t)last_pos / C_next - nb0 + 1) : 0;
        const bool local_nh = nh.bits > 0 && span <= EMIT_SPAN;
        if (local_nh)
            for (int k = threadIdx.x; k < RS_RADIX_MAX * EMIT_SPAN; k += EMIT_THREADS) (&s_nh[0][0])[k] = 0u;
        __syncthreads();
        // thread i emits the contiguous instances [i P, (i + 1) P) of a range
        // of the round: one search for its first row, then a walk along the
        // rects.  A round of few instances per thread writes them directly
        // (neighbouring threads' runs are close together); a larger one goes
        // in chunks of EMIT_STAGE through shared memory and the block writes
        // each chunk out with coalesced stores.
        auto walk = [&](uint32_t k, uint32_t kend, uint32_t c0, bool staged) {
            int a = 0, b = rows - 1;                 // last row j with s_off[j] <= k
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (s_off[mid] <= k) a = mid;
                else b = mid - 1;
            }
            uint32_t off = k - s_off[a];
            short4 r = s_rect[a];
            uint32_t g = s_row[a];
            int v = view_of(g);
            uint32_t t0 = s_tileoff[v];
            int gx = s_gx[v];
            uint32_t wdt = (uint32_t)(r.z - r.x + 1);
            int ty = r.y + (int)(off / wdt), tx = r.x + (int)(off % wdt);
            uint32_t row_end = a + 1 < rows ? s_off[a + 1] : total;
            // next-pass block of the current position, advanced incrementally
            // (positions grow by one per instance)
            uint32_t nb = (uint32_t)(base + k) / C_next;
            uint64_t nb_end = (uint64_t)(nb + 1) * C_next;
            for (; k < kend; ++k) {
                while (k >= row_end) {               // next row (every visible row has instances)
                    ++a;
                    r = s_rect[a];
                    g = s_row[a];
                    v = view_of(g);
                    t0 = s_tileoff[v];
                    gx = s_gx[v];
                    ty = r.y;
                    tx = r.x;
                    row_end = a + 1 < rows ? s_off[a + 1] : total;
                }
                const int64_t pos = base + k;
                if (pos >= cap) break;
                const uint32_t t = t0 + (uint32_t)(ty * gx + tx);
                if (STAGED && staged) {
                    s_et[k - c0] = t;
                    s_eg[k - c0] = g;
                } else {
                    inst_tile[pos] = t;
                    inst_gid[pos] = g;
                }
                if ((uint64_t)pos >= nb_end) {
                    ++nb;
                    nb_end += C_next;
                }
                if (local_nh)
                    atomicAdd(&s_nh[(t >> nh.shift) & nmask][nb - nb0], 1u);
                else if (nh.bits > 0)
                    atomicAdd(nh.hist + (size_t)((t >> nh.shift) & nmask) * nh.G + nb, 1u);
                if (++tx > r.z) {
                    tx = r.x;
                    ++ty;
                }
            }
        };
        if (!STAGED || total <= EMIT_DIRECT_MAX) {
            const uint32_t P = (total + EMIT_THREADS - 1) / EMIT_THREADS;
            const uint32_t k = threadIdx.x * P;
            if (k < total) walk(k, min(total, k + P), 0u, false);
        } else {
            for (uint32_t c0 = 0; c0 < total; c0 += EMIT_STAGE) {
                const uint32_t cn = min((uint32_t)EMIT_STAGE, total - c0);
                const uint32_t P = (cn + EMIT_THREADS - 1) / EMIT_THREADS;
                const uint32_t k = c0 + threadIdx.x * P;
                if (k < c0 + cn) walk(k, min(c0 + cn, k + P), c0, true);
                __syncthreads();
                for (uint32_t j = threadIdx.x; j < cn; j += EMIT_THREADS) {
                    const int64_t pos = base + c0 + j;
                    if (pos < cap) {
                        inst_tile[pos] = s_et[j];
                        inst_gid[pos] = s_eg[j];
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();
        if (local_nh)
            for (int k = threadIdx.x; k < (1 << nh.bits) * span; k += EMIT_THREADS) {
                const int d = k / span, j = k - d * span;
                const uint32_t h = s_nh[d][j];
                if (h) atomicAdd(nh.hist + (size_t)d * nh.G + (size_t)(nb0 + j), h);
            }
        base += total;
        __syncthreads();
    }
}

// Tile schedule: every tile id once, longest lists first.  Class of a tile:
// its list length in quarter octaves, 4 clz(length) + 3 - (the two bits below
// the leading one), 0 .. 127 from the longest lists down, 128 for empty
// tiles.  A stable counting sort by class in one block: warp w owns the
// contiguous tiles [w C, (w + 1) C) and walks them 32 at a time, ranking equal
// classes with __match_any_sync; per-warp class counts, their prefix in
// (class, warp) order, then a second walk writes every tile at its place.
constexpr int TO_THREADS = 1024;
constexpr int TO_WARPS = TO_THREADS / 32;
constexpr int TO_CLASSES = 129;

__device__ __forceinline__ int tile_class(uint2 r) {
    const uint32_t len = r.y - r.x;
    if (!len) return TO_CLASSES - 1;
    const int z = __clz(len);
    const uint32_t next2 = z <= 29 ? (len << (z + 1)) >> 30 : (z == 30 ? ((len & 1u) << 1) : 0u);
    return 4 * z + 3 - (int)next2;
}

__global__ void __launch_bounds__(TO_THREADS) tile_order_kernel(const uint2* __restrict__ ranges, int T,
                                                                uint32_t* __restrict__ order) {
    pdl_wait_and_trigger();
    __shared__ uint32_t s_cnt[TO_WARPS][TO_CLASSES];
    __shared__ uint32_t s_tot[TO_CLASSES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < TO_WARPS * TO_CLASSES; k += TO_THREADS) (&s_cnt[0][0])[k] = 0u;
    __syncthreads();
    const int C = (T + TO_WARPS - 1) / TO_WARPS;
    const int lo = warp * C, hi = min(T, lo + C);
    const unsigned lt = (1u << lane) - 1u;
    for (int b = lo; b < hi; b += 32) {                  // per-warp class counts
        const int t = b + lane;
        const int c = t < hi ? tile_class(ranges[t]) : TO_CLASSES;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c < TO_CLASSES && (peers & lt) == 0u) s_cnt[warp][c] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < TO_CLASSES) {
        uint32_t tot = 0;
        for (int w = 0; w < TO_WARPS; ++w) tot += s_cnt[w][threadIdx.x];
        s_tot[threadIdx.x] = tot;
    }
    __syncthreads();
    if (warp == 0) {                                    // exclusive scan of the class totals
        constexpr int PER = (TO_CLASSES + 31) / 32;
        uint32_t v[PER], mine = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int c = lane * PER + q;
            v[q] = c < TO_CLASSES ? s_tot[c] : 0u;
            mine += v[q];
        }
        uint32_t x = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        uint32_t run = x - mine;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int c = lane * PER + q;
            if (c < TO_CLASSES) s_tot[c] = run;
            run += v[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < TO_CLASSES) {                     // place of each (class, warp) run
        uint32_t run = s_tot[threadIdx.x];
        for (int w = 0; w < TO_WARPS; ++w) {
            const uint32_t n = s_cnt[w][threadIdx.x];
            s_cnt[w][threadIdx.x] = run;
            run += n;
        }
    }
    __syncthreads();
    for (int b = lo; b < hi; b += 32) {                  // same walk: write every tile at its place
        const int t = b + lane;
        const int c = t < hi ? tile_class(ranges[t]) : TO_CLASSES;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c < TO_CLASSES) order[s_cnt[warp][c] + (uint32_t)__popc(peers & lt)] = (uint32_t)t;
        __syncwarp();
        if (c < TO_CLASSES && (peers & lt) == 0u) s_cnt[warp][c] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

static cudaError_t launch_tile_order(const sgs_bins& out, int T, bool pdl, cudaStream_t stream) {
    if (!out.order || T <= 0) return cudaGetLastError();
    (void)launch_pdl_if(pdl, tile_order_kernel, dim3(1), dim3(TO_THREADS), 0, stream,
                        reinterpret_cast<const uint2*>(out.ranges), T, out.order);
    note_launch();
    return cudaGetLastError();
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tile_sorted, const int32_t* d_n, int64_t cap,
                              uint2* __restrict__ ranges) {
    pdl_wait_and_trigger();
    int64_t n = read_n(d_n, 0, cap);
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t t = tile_sorted[k];
        if (k == 0 || tile_sorted[k - 1] != t) ranges[t].x = (uint32_t)k;
        if (k == n - 1 || tile_sorted[k + 1] != t) ranges[t].y = (uint32_t)(k + 1);
    }
}

__global__ void keys_kernel(const uint32_t* __restrict__ tile_sorted, const uint32_t* __restrict__ gids,
                            const float* __restrict__ depth, const int32_t* d_n, int64_t cap,
                            uint64_t* __restrict__ keys) {
    pdl_wait_and_trigger();
    int64_t n = read_n(d_n, 0, cap);
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k < n; k += (int64_t)gridDim.x * blockDim.x)
        keys[k] = ((uint64_t)tile_sorted[k] << 32) | (uint64_t)__float_as_uint(depth[gids[k]]);
}

static int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

struct TileSortCfg {
    int bits, passes, bits_per;
};

static TileSortCfg tile_sort_cfg(int num_tiles) {
    TileSortCfg c;
    c.bits = ceil_log2(num_tiles);
    c.passes = (c.bits + RS_MAX_BITS - 1) / RS_MAX_BITS;
    c.bits_per = c.passes ? (c.bits + c.passes - 1) / c.passes : 0;
    return c;
}

struct SortGeom {
    int G_depth, G_emit, G_tile;
    TileSortCfg tc;
};

static SortGeom sort_geom(int n, int64_t cap, int num_tiles) {
    SortGeom g;
    g.G_depth = sort_blocks(n, RS_TILE);
    int64_t ge = ((int64_t)n + EMIT_ROWS_PER_BLOCK - 1) / EMIT_ROWS_PER_BLOCK;
    g.G_emit = (int)(ge < 1 ? 1 : (ge > EMIT_G_MAX ? EMIT_G_MAX : ge));
    g.G_tile = sort_blocks(cap, RS_TILE);
    g.tc = tile_sort_cfg(num_tiles > 0 ? num_tiles : 1);
    return g;
}

struct BinWs {
    uint32_t *dkey[2], *perm[2], *cnt, *inst_tile[2], *inst_gid_tmp;
    // zeroed at the start of every sort (histograms built with atomics):
    uint32_t* depth_hist;     // [DEPTH_PASSES][256][G_depth]
    uint32_t* depth_tot;      // [DEPTH_PASSES][256]
    uint32_t* tile_hist;      // [TILE_PASSES_MAX][256][G_tile]
    uint32_t* tile_tot;       // [TILE_PASSES_MAX][256]
    unsigned long long* esum; // [G_emit]
    size_t zero_bytes;
    size_t bytes;
};

static BinWs carve_bin_ws(void* base, int n, int64_t cap, int num_tiles) {
    Carver c{reinterpret_cast<char*>(base), 0};
    BinWs w;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t cc = (size_t)(cap > 0 ? cap : 1);
    const SortGeom sg = sort_geom(n, cap, num_tiles);
    w.dkey[0] = c.take<uint32_t>(nn);
    w.dkey[1] = c.take<uint32_t>(nn);
    w.perm[0] = c.take<uint32_t>(nn);
    w.perm[1] = c.take<uint32_t>(nn);
    w.cnt = c.take<uint32_t>(nn);
    w.inst_tile[0] = c.take<uint32_t>(cc);
    w.inst_tile[1] = c.take<uint32_t>(cc);
    w.inst_gid_tmp = c.take<uint32_t>(cc);
    c.off = align_up(c.off, 256);
    const size_t z0 = c.off;
    w.depth_hist = c.take<uint32_t>((size_t)DEPTH_PASSES * RS_RADIX_MAX * sg.G_depth);
    w.depth_tot = c.take<uint32_t>((size_t)DEPTH_PASSES * RS_RADIX_MAX);
    w.tile_hist = c.take<uint32_t>((size_t)TILE_PASSES_MAX * RS_RADIX_MAX * sg.G_tile);
    w.tile_tot = c.take<uint32_t>((size_t)TILE_PASSES_MAX * RS_RADIX_MAX);
    w.esum = c.take<unsigned long long>((size_t)sg.G_emit);
    w.zero_bytes = c.off - z0;
    w.bytes = c.off + 256;
    return w;
}

size_t bin_sort_ws_bytes(int n, int64_t capacity, int num_tiles) {
    return carve_bin_ws(nullptr, n, capacity, num_tiles).bytes;
}

cudaError_t launch_bin_sort(const sgs_proj& proj, const ViewsDev& vd, const SetDev& st, const sgs_bins& out, void* ws,
                            cudaStream_t stream) {
    (void)st;
    const int n = vd.row_off[vd.nv];            // projection rows
    // dependent launches between the sort's kernels measured faster up to a
    // few million rows (one view) and slower on the multi-view sorts of tens
    // of millions of rows, so they are used up to kSortPdlMaxRows
    const bool pdl = n <= kSortPdlMaxRows;
    const int T = vd.T_total;
    BinWs w = carve_bin_ws(ws, n, out.capacity, T);
    const SortGeom sg = sort_geom(n, out.capacity, T);
    const TileSortCfg& tc = sg.tc;
    cudaError_t e = cudaMemsetAsync(out.ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, stream);
    if (e != cudaSuccess) return e;
    if (n == 0) {
        e = cudaMemsetAsync(out.count, 0, sizeof(int32_t), stream);
        return e != cudaSuccess ? e : launch_tile_order(out, T, pdl, stream);
    }
    e = cudaMemsetAsync(w.depth_hist, 0, w.zero_bytes, stream);
    if (e != cudaSuccess) return e;
    auto depth_pass = [&](int p) {
        return PassDesc{8 * p, 8, w.depth_hist + (size_t)p * RS_RADIX_MAX * sg.G_depth,
                        w.depth_tot + p * RS_RADIX_MAX, sg.G_depth};
    };
    auto tile_pass = [&](int p) {
        const int bits = min(tc.bits_per, tc.bits - p * tc.bits_per);
        return PassDesc{p * tc.bits_per, bits, w.tile_hist + (size_t)p * RS_RADIX_MAX * sg.G_tile,
                        w.tile_tot + p * RS_RADIX_MAX, sg.G_tile};
    };
    const NextHist none{0, 0, nullptr, 1};
    // 1. stable sort of the visible rows by depth bits (4 passes of 8 bits; the
    //    first pass drops the rows that touch no tile, the last one also
    //    gathers the rows' tile counts in depth order)
    (void)launch_pdl_if(pdl, depth_hist_first_kernel, dim3(sg.G_depth), dim3(RS_THREADS), 0, stream, proj.depth,
                        proj.tiles_touched, n, depth_pass(0));
    note_launch();
    for (int p = 0; p < DEPTH_PASSES; ++p) {
        const PassDesc ps = depth_pass(p);
        const int src = (p + 1) & 1, dst = p & 1;     // pass 0 -> buffer 0 -> 1 -> 0 -> 1
        if (p > 0) {
            (void)launch_pdl_if(pdl, pass_hist_kernel, dim3(sg.G_depth), dim3(RS_THREADS), 0, stream, w.dkey[src],
                                depth_pass(p - 1).tot, RS_RADIX_MAX, ps);
            note_launch();
        }
        (void)launch_pdl_if(pdl, pass_scan_kernel, dim3(1 << ps.bits), dim3(SORT_G_MAX), 0, stream, ps.hist, ps.G,
                            ps.tot);
        note_launch();
        const bool last = p + 1 == DEPTH_PASSES;
        uint32_t* kout = last ? nullptr : w.dkey[dst];
        if (p == 0)
            (void)launch_pdl_if(pdl, pass_scatter_kernel<true, false>, dim3(sg.G_depth), dim3(RS_THREADS), 0, stream,
                                nullptr, nullptr, proj.depth, proj.tiles_touched, n, kout, w.perm[dst], ps, nullptr,
                                nullptr, 1);
        else if (!last)
            (void)launch_pdl_if(pdl, pass_scatter_kernel<false, false>, dim3(sg.G_depth), dim3(RS_THREADS), 0, stream,
                                w.dkey[src], w.perm[src], nullptr, nullptr, 0, kout, w.perm[dst], ps, nullptr,
                                nullptr, 1);
        else
            (void)launch_pdl_if(pdl, pass_scatter_kernel<false, true>, dim3(sg.G_depth), dim3(RS_THREADS), 0, stream,
                                w.dkey[src], w.perm[src], nullptr, proj.tiles_touched, 0, kout, w.perm[dst], ps,
                                w.cnt, w.esum, sg.G_emit);
        note_launch();
    }
    const uint32_t* perm = w.perm[(DEPTH_PASSES - 1) & 1];
    // 2. instance offsets (M) and load-balanced emission in depth order; the
    //    tile sort's result must land in out.gids, so pick the starting buffer
    //    by the pass parity.
    uint32_t* gk[2] = {w.inst_tile[0], w.inst_tile[1]};
    uint32_t* gv[2];
    if (tc.passes % 2 == 0) {
        gv[0] = out.gids;
        gv[1] = w.inst_gid_tmp;
    } else {
        gv[0] = w.inst_gid_tmp;
        gv[1] = out.gids;
    }
    (void)launch_pdl_if(pdl, emit_offsets_kernel, dim3(1), dim3(SORT_G_MAX), 0, stream, w.esum, sg.G_emit, out.count);
    note_launch();
    {
        NextHist nh = none;
        if (tc.passes > 0) {
            const PassDesc q = tile_pass(0);
            nh = NextHist{q.shift, q.bits, q.hist, q.G};
        }
        // blocks of many rows (the emission grid at its cap) stage their
        // instances for coalesced writes; short blocks write directly
        const bool staged = (int64_t)n > (int64_t)EMIT_G_MAX * EMIT_ROWS_PER_BLOCK;
        (void)launch_pdl_if(pdl, staged ? emit_kernel<true> : emit_kernel<false>, dim3(sg.G_emit),
                            dim3(EMIT_THREADS), 0, stream, perm, w.cnt,
                            reinterpret_cast<const short4*>(proj.rect), w.depth_tot, vd, out.capacity, w.esum,
                            sg.G_emit, out.count, gk[0], gv[0], nh);
        note_launch();
    }
    // 3. stable passes over the written instances by tile id (the first
    //    pass's counts come from the emission)
    for (int p = 0; p < tc.passes; ++p) {
        const PassDesc ps = tile_pass(p);
        if (p > 0) {
            const PassDesc q = tile_pass(p - 1);
            (void)launch_pdl_if(pdl, pass_hist_kernel, dim3(sg.G_tile), dim3(RS_THREADS), 0, stream, gk[p & 1], q.tot,
                                1 << q.bits, ps);
            note_launch();
        }
        (void)launch_pdl_if(pdl, pass_scan_kernel, dim3(1 << ps.bits), dim3(SORT_G_MAX), 0, stream, ps.hist, ps.G,
                            ps.tot);
        note_launch();
        (void)launch_pdl_if(pdl, pass_scatter_kernel<false, false>, dim3(sg.G_tile), dim3(RS_THREADS), 0, stream,
                            gk[p & 1], gv[p & 1], nullptr, nullptr, 0, gk[(p + 1) & 1], gv[(p + 1) & 1], ps, nullptr,
                            nullptr, 1);
        note_launch();
    }
    const uint32_t* tile_sorted = gk[tc.passes & 1];
    // 4. per-tile ranges and optional 64-bit keys
    const int rb = 152 * 8;
    (void)launch_pdl_if(pdl, ranges_kernel, dim3(rb), dim3(256), 0, stream, tile_sorted, out.count, out.capacity,
                        reinterpret_cast<uint2*>(out.ranges));
    note_launch();
    if (out.keys) {
        (void)launch_pdl_if(pdl, keys_kernel, dim3(rb), dim3(256), 0, stream, tile_sorted, out.gids, proj.depth,
                            out.count, out.capacity, out.keys);
        note_launch();
    }
    return launch_tile_order(out, T, pdl, stream);
}

}  // namespace sgs
