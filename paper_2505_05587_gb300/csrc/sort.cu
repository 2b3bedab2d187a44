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
    __shared__ uint32_t s_warp[32];
    uint32_t v = threadIdx.x < nb ? partial[threadIdx.x] : 0u;
    uint32_t inc = block_inclusive_scan(v, s_warp);
    if (threadIdx.x < nb) partial[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1 && d_total) *d_total = inc;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_downsweep_kernel(
    const uint32_t* __restrict__ in, uint32_t* __restrict__ out, const int32_t* d_n, int64_t n_max,
    const uint32_t* __restrict__ partial) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    int64_t n = read_n(d_n, n_max, n_max);
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
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
    scan_reduce_kernel<<<nb, SCAN_THREADS, 0, stream>>>(in, d_n, n_max, partial);
    note_launch();
    scan_partials_kernel<<<1, SCAN_THREADS, 0, stream>>>(partial, nb, d_total);
    note_launch();
    scan_downsweep_kernel<<<nb, SCAN_THREADS, 0, stream>>>(in, out, d_n, n_max, partial);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value) pairs.
// Each of G blocks owns one contiguous chunk of the items.
// Per pass: per-block digit histogram -> per-digit exclusive scan over blocks
// -> stable scatter.  Inside a block, ranks come from warp-level
// __match_any_sync over 32 consecutive items, accumulated across sub-rounds
// and across warps in item order, which keeps equal digits in input order.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_MAX_BITS = 8;
constexpr int RS_RADIX_MAX = 1 << RS_MAX_BITS;
constexpr int RS_MAX_BLOCKS = 1024;

// Up to RS_MAX_BLOCKS blocks; each owns a contiguous chunk rounded only to
// whole warps, so that the device-side count n (often far below n_max) still
// spreads over every block and each SM keeps several blocks in flight.
static int rs_blocks(int64_t n_max) {
    int64_t b = (n_max + 255) / 256;
    if (b < 1) b = 1;
    if (b > RS_MAX_BLOCKS) b = RS_MAX_BLOCKS;
    return (int)b;
}

__device__ __forceinline__ void rs_chunk(int64_t n, int64_t* start, int64_t* end) {
    int64_t per = (n + gridDim.x - 1) / gridDim.x;
    per = (per + 31) / 32 * 32;
    *start = (int64_t)blockIdx.x * per;
    *end = min(n, *start + per);
}

__global__ void __launch_bounds__(RS_THREADS) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                const int32_t* d_n, int64_t n_host,
                                                                int64_t cap, int shift, int bits,
                                                                uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_cnt[RS_RADIX_MAX];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    for (int d = threadIdx.x; d < radix; d += blockDim.x) s_cnt[d] = 0;
    __syncthreads();
    int64_t n = read_n(d_n, n_host, cap), start, end;
    rs_chunk(n, &start, &end);
    const int lane = threadIdx.x & 31;
    for (int64_t base = start; base < end; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        bool valid = i < end;
        uint32_t d = valid ? ((keys[i] >> shift) & mask) : (uint32_t)radix;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&s_cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[(size_t)d * gridDim.x + blockIdx.x] = s_cnt[d];
}

// One block per digit: exclusive scan of that digit's counts over the G blocks.
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* __restrict__ hist, int G,
                                                          uint32_t* __restrict__ digit_tot) {
    __shared__ uint32_t s_warp[32];
    uint32_t* h = hist + (size_t)blockIdx.x * G;
    uint32_t v = threadIdx.x < G ? h[threadIdx.x] : 0u;
    uint32_t inc = block_inclusive_scan(v, s_warp);
    if (threadIdx.x < G) h[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1) digit_tot[blockIdx.x] = inc;
}

__global__ void __launch_bounds__(RS_THREADS) radix_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int32_t* d_n,
    int64_t n_host, int64_t cap, int shift, int bits, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ digit_tot) {
    __shared__ uint32_t s_warp[RS_WARPS][RS_RADIX_MAX + 1];
    __shared__ uint32_t s_off[RS_RADIX_MAX];
    __shared__ uint32_t s_tot[RS_RADIX_MAX];
    __shared__ uint32_t s_scan[32];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // digit base = exclusive scan of the digit totals (radix <= RS_THREADS)
    {
        uint32_t v = threadIdx.x < radix ? digit_tot[threadIdx.x] : 0u;
        // block_inclusive_scan assumes <= 32 warps; RS_THREADS = 256
        uint32_t inc;
        {
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            if (lane == 31) s_scan[warp] = x;
            __syncthreads();
            if (warp == 0) {
                uint32_t w = lane < RS_WARPS ? s_scan[lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += t;
                }
                s_scan[lane] = w;
            }
            __syncthreads();
            inc = x + (warp > 0 ? s_scan[warp - 1] : 0u);
        }
        if (threadIdx.x < radix)
            s_off[threadIdx.x] = (inc - v) + hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
    }
    __syncthreads();

    int64_t n = read_n(d_n, n_host, cap), start, end;
    rs_chunk(n, &start, &end);
    for (int64_t tile = start; tile < end; tile += RS_TILE) {
        for (int k = threadIdx.x; k < RS_WARPS * (RS_RADIX_MAX + 1); k += RS_THREADS)
            (&s_warp[0][0])[k] = 0u;
        __syncthreads();
        uint32_t key[RS_ITEMS], val[RS_ITEMS], dig[RS_ITEMS], rank[RS_ITEMS];
        const int64_t wbase = tile + (int64_t)warp * 32 * RS_ITEMS + lane;
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            int64_t idx = wbase + it * 32;
            bool valid = idx < end;
            key[it] = valid ? keys_in[idx] : 0u;
            val[it] = valid ? vals_in[idx] : 0u;
            dig[it] = valid ? ((key[it] >> shift) & mask) : (uint32_t)radix;
        }
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            unsigned peers = __match_any_sync(0xffffffffu, dig[it]);
            unsigned lower = peers & ((1u << lane) - 1u);
            uint32_t base = s_warp[warp][dig[it]];
            rank[it] = base + (uint32_t)__popc(lower);
            __syncwarp();
            if (lower == 0u) s_warp[warp][dig[it]] = base + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < radix; d += RS_THREADS) {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = s_warp[w][d];
                s_warp[w][d] = sum;
                sum += c;
            }
            s_tot[d] = sum;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            if (dig[it] < (uint32_t)radix) {
                uint32_t dest = s_off[dig[it]] + s_warp[warp][dig[it]] + rank[it];
                keys_out[dest] = key[it];
                vals_out[dest] = val[it];
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < radix; d += RS_THREADS) s_off[d] += s_tot[d];
        __syncthreads();
    }
}

struct RadixBufs {
    uint32_t* hist;       // [RS_RADIX_MAX * RS_MAX_BLOCKS]
    uint32_t* digit_tot;  // [RS_RADIX_MAX]
};

static int rs_passes(int total_bits) { return (total_bits + RS_MAX_BITS - 1) / RS_MAX_BITS; }

// Sorts (k[0], v[0]) using (k[1], v[1]) as the ping-pong pair; the result is
// in pair (passes % 2).  Bits [0, total_bits) are sorted.
static cudaError_t radix_sort_pairs(uint32_t* k[2], uint32_t* v[2], const int32_t* d_n, int64_t n_host,
                                    int64_t n_max, int total_bits, const RadixBufs& rb,
                                    cudaStream_t stream) {
    if (total_bits <= 0) return cudaSuccess;
    int G = rs_blocks(n_max);
    int passes = rs_passes(total_bits);
    int bits_per = (total_bits + passes - 1) / passes;
    int shift = 0;
    for (int p = 0; p < passes; ++p) {
        int bits = min(bits_per, total_bits - shift);
        int src = p & 1, dst = src ^ 1;
        radix_hist_kernel<<<G, RS_THREADS, 0, stream>>>(k[src], d_n, n_host, n_max, shift, bits, rb.hist);
        note_launch();
        radix_scan_kernel<<<1 << bits, 1024, 0, stream>>>(rb.hist, G, rb.digit_tot);
        note_launch();
        radix_scatter_kernel<<<G, RS_THREADS, 0, stream>>>(k[src], v[src], k[dst], v[dst], d_n, n_host,
                                                           n_max, shift, bits, rb.hist, rb.digit_tot);
        note_launch();
        shift += bits;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Binning kernels
// ---------------------------------------------------------------------------
__global__ void visible_flags_kernel(const uint32_t* __restrict__ tiles, int n, uint32_t* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = tiles[i] ? 1u : 0u;
}

// Compacts the visible Gaussians (in index order) into (depth bits, index)
// pairs.  depth > near_z > 0 for every visible Gaussian, so its bits order like
// the value.
__global__ void depth_keys_kernel(const float* __restrict__ depth, const uint32_t* __restrict__ tiles,
                                  const uint32_t* __restrict__ pos, int n, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tiles[i] == 0u) return;
    const uint32_t p = pos[i];
    keys[p] = __float_as_uint(depth[i]);
    vals[p] = (uint32_t)i;
}

__global__ void gather_counts_kernel(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ tiles,
                                     const int32_t* __restrict__ d_n, int n_max, uint32_t* __restrict__ cnt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_max) return;
    cnt[j] = j < *d_n ? tiles[perm[j]] : 0u;
}

// One thread per depth-sorted projection row: writes the row's instances
// (global tile id in the row's view, row) in row-major tile order.
__global__ void emit_kernel(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cnt,
                            const uint32_t* __restrict__ offs, const short4* __restrict__ rect, int n_rows,
                            ViewsDev vd, int64_t cap, uint32_t* __restrict__ inst_tile,
                            uint32_t* __restrict__ inst_gid) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_rows) return;
    uint32_t c = cnt[j];
    if (c == 0) return;
    uint32_t g = perm[j];
    const int v = view_of_row(vd, g);
    const int gx = vd.cam[v].gx;
    const uint32_t t0 = (uint32_t)vd.tile_off[v];
    short4 r = rect[g];
    int64_t pos = offs[j];
    for (int ty = r.y; ty <= r.w; ++ty)
        for (int tx = r.x; tx <= r.z; ++tx) {
            if (pos < cap) {
                inst_tile[pos] = t0 + (uint32_t)(ty * gx + tx);
                inst_gid[pos] = g;
            }
            ++pos;
        }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tile_sorted, const int32_t* d_n, int64_t cap,
                              uint2* __restrict__ ranges) {
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

struct BinWs {
    uint32_t *dkey[2], *perm[2], *cnt, *offs, *inst_tile[2], *inst_gid_tmp, *n_vis;
    void* scan_tmp;
    RadixBufs rb;
    size_t bytes;
};

static BinWs carve_bin_ws(void* base, int n, int64_t cap) {
    Carver c{reinterpret_cast<char*>(base), 0};
    BinWs w;
    size_t nn = (size_t)(n > 0 ? n : 1);
    size_t cc = (size_t)(cap > 0 ? cap : 1);
    w.dkey[0] = c.take<uint32_t>(nn);
    w.dkey[1] = c.take<uint32_t>(nn);
    w.perm[0] = c.take<uint32_t>(nn);
    w.perm[1] = c.take<uint32_t>(nn);
    w.cnt = c.take<uint32_t>(nn);
    w.offs = c.take<uint32_t>(nn);
    w.inst_tile[0] = c.take<uint32_t>(cc);
    w.inst_tile[1] = c.take<uint32_t>(cc);
    w.inst_gid_tmp = c.take<uint32_t>(cc);
    w.n_vis = c.take<uint32_t>(1);
    w.scan_tmp = c.take<char>(scan_tmp_bytes(n));
    w.rb.hist = c.take<uint32_t>((size_t)RS_RADIX_MAX * RS_MAX_BLOCKS);
    w.rb.digit_tot = c.take<uint32_t>(RS_RADIX_MAX);
    w.bytes = c.off + 256;
    return w;
}

size_t bin_sort_ws_bytes(int n, int64_t capacity, int num_tiles) {
    (void)num_tiles;
    return carve_bin_ws(nullptr, n, capacity).bytes;
}

cudaError_t launch_bin_sort(const sgs_proj& proj, const ViewsDev& vd, const SetDev& st, const sgs_bins& out, void* ws,
                            cudaStream_t stream) {
    (void)st;
    const int n = vd.row_off[vd.nv];            // projection rows
    BinWs w = carve_bin_ws(ws, n, out.capacity);
    const int T = vd.T_total;
    cudaError_t e = cudaMemsetAsync(out.ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, stream);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaMemsetAsync(out.count, 0, sizeof(int32_t), stream);
    const int nb = (n + 255) / 256;
    const int32_t* d_nvis = reinterpret_cast<const int32_t*>(w.n_vis);
    // 1. compact the visible Gaussians, then a stable sort of them by depth bits
    visible_flags_kernel<<<nb, 256, 0, stream>>>(proj.tiles_touched, n, w.cnt);
    note_launch();
    e = launch_exclusive_scan(w.cnt, w.offs, w.n_vis, n, nullptr, w.scan_tmp, stream);
    if (e != cudaSuccess) return e;
    depth_keys_kernel<<<nb, 256, 0, stream>>>(proj.depth, proj.tiles_touched, w.offs, n, w.dkey[0], w.perm[0]);
    note_launch();
    e = radix_sort_pairs(w.dkey, w.perm, d_nvis, 0, n, 32, w.rb, stream);
    if (e != cudaSuccess) return e;
    const uint32_t* perm = w.perm[rs_passes(32) & 1];
    // 2. instance offsets in depth order, M
    gather_counts_kernel<<<nb, 256, 0, stream>>>(perm, proj.tiles_touched, d_nvis, n, w.cnt);
    note_launch();
    e = launch_exclusive_scan(w.cnt, w.offs, reinterpret_cast<uint32_t*>(out.count), n, nullptr,
                              w.scan_tmp, stream);
    if (e != cudaSuccess) return e;
    // 3. emit (tile, gid) instances in depth order; the tile sort's result must
    //    land in out.gids, so pick the starting buffer by the pass parity.
    const int tile_bits = ceil_log2(T);
    const int tpasses = rs_passes(tile_bits);
    uint32_t* gk[2];
    uint32_t* gv[2];
    gk[0] = w.inst_tile[0];
    gk[1] = w.inst_tile[1];
    if (tpasses % 2 == 0) {
        gv[0] = out.gids;
        gv[1] = w.inst_gid_tmp;
    } else {
        gv[0] = w.inst_gid_tmp;
        gv[1] = out.gids;
    }
    emit_kernel<<<nb, 256, 0, stream>>>(perm, w.cnt, w.offs, reinterpret_cast<const short4*>(proj.rect), n, vd,
                                        out.capacity, gk[0], gv[0]);
    note_launch();
    // 4. stable sort of the instances by tile id
    e = radix_sort_pairs(gk, gv, out.count, 0, out.capacity, tile_bits, w.rb, stream);
    if (e != cudaSuccess) return e;
    const uint32_t* tile_sorted = gk[tpasses & 1];
    // 5. per-tile ranges and optional 64-bit keys
    int rb = 152 * 8;
    ranges_kernel<<<rb, 256, 0, stream>>>(tile_sorted, out.count, out.capacity,
                                          reinterpret_cast<uint2*>(out.ranges));
    note_launch();
    if (out.keys)
        keys_kernel<<<rb, 256, 0, stream>>>(tile_sorted, out.gids, proj.depth, out.count, out.capacity,
                                            out.keys);
        note_launch();
    return cudaGetLastError();
}

}  // namespace sgs
