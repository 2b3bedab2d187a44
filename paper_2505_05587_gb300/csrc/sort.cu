// Tile binning and depth sort (Section 3: "sorts points according to
// view-dependent depth" before alpha compositing).
//
// Order produced: instances (row r, tile t) sorted by (t, float32 depth bits
// of r, r), where a row is a (view, Gaussian) pair of the projection.
// Design: a most-significant-digit pass of a radix sort on the tile id -- a
// counting sort: per-tile counts, their exclusive scan (the per-tile ranges),
// and emission of every instance into its tile's bucket -- followed by one CTA
// per tile sorting its bucket by the 64-bit key (depth bits << 32 | row) in
// shared memory (bitonic network; buckets longer than shared memory are sorted
// in shared-memory chunks that the same CTA then merges).  The keys are
// distinct, so the order is total and identical to one stable sort of
// (tile << 32 | depth bits) over instances emitted in row order.
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
// Binning kernels
// ---------------------------------------------------------------------------
// Per-tile counters live one per 128-byte line (stride kPad words) so that the
// atomics of different tiles do not serialise on shared cache lines.
constexpr int kPad = 32;

__global__ void tile_count_kernel(const short4* __restrict__ rect, const uint32_t* __restrict__ tiles, int n_rows,
                                  ViewsDev vd, uint32_t* __restrict__ tile_cnt_pad) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows || tiles[r] == 0u) return;
    const int v = view_of_row(vd, r);
    const int gx = vd.cam[v].gx;
    const int t0 = vd.tile_off[v];
    const short4 b = rect[r];
    for (int ty = b.y; ty <= b.w; ++ty)
        for (int tx = b.x; tx <= b.z; ++tx) atomicAdd(&tile_cnt_pad[(size_t)(t0 + ty * gx + tx) * kPad], 1u);
}

__global__ void unpad_kernel(const uint32_t* __restrict__ pad, int T, uint32_t* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) out[t] = pad[(size_t)t * kPad];
}

__global__ void emit_kernel(const short4* __restrict__ rect, const uint32_t* __restrict__ tiles,
                            const float* __restrict__ depth, int n_rows, ViewsDev vd,
                            const uint32_t* __restrict__ tile_start, uint32_t* __restrict__ tile_fill, int64_t cap,
                            uint64_t* __restrict__ bucket) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows || tiles[r] == 0u) return;
    const int v = view_of_row(vd, r);
    const int gx = vd.cam[v].gx;
    const int t0 = vd.tile_off[v];
    // depth > near_z > 0 for every visible row, so its bits order like the value
    const uint64_t key = ((uint64_t)__float_as_uint(depth[r]) << 32) | (uint64_t)(uint32_t)r;
    const short4 b = rect[r];
    for (int ty = b.y; ty <= b.w; ++ty)
        for (int tx = b.x; tx <= b.z; ++tx) {
            const int t = t0 + ty * gx + tx;
            const int64_t pos = (int64_t)tile_start[t] + atomicAdd(&tile_fill[(size_t)t * kPad], 1u);
            if (pos < cap) bucket[pos] = key;
        }
}

constexpr int TS_THREADS = 256;
constexpr int TS_CAP = 4096;          // keys sorted at once in shared memory (32 KB)

// Ascending bitonic sort of s[0, P) in shared memory (P a power of two).
__device__ __forceinline__ void bitonic_sort_smem(uint64_t* s, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int idx = threadIdx.x; idx < (P >> 1); idx += blockDim.x) {
                const int i = 2 * idx - (idx & (j - 1));
                const int p = i + j;
                const uint64_t a = s[i], b = s[p];
                const bool up = (i & k) == 0;
                if ((a > b) == up) {
                    s[i] = b;
                    s[p] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Sorts keys[0, L) of one tile into out[0, L) (keys may be reordered).
// Runs of TS_CAP are sorted in shared memory, then merged pairwise by the CTA
// (merge path: each thread finds its output range by binary search, then
// merges serially), ping-ponging between the two buffers.
__device__ void sort_segment(uint64_t* keys, uint64_t* tmp, int L, uint64_t* s, uint64_t** result) {
    for (int c = 0; c < L; c += TS_CAP) {
        const int n = min(TS_CAP, L - c);
        int P = 1;
        while (P < n) P <<= 1;
        for (int k = threadIdx.x; k < P; k += blockDim.x) s[k] = k < n ? keys[c + k] : ~0ull;
        __syncthreads();
        bitonic_sort_smem(s, P);
        for (int k = threadIdx.x; k < n; k += blockDim.x) keys[c + k] = s[k];
        __syncthreads();
    }
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int run = TS_CAP; run < L; run <<= 1) {
        for (int a0 = 0; a0 < L; a0 += 2 * run) {
            const int na = min(run, L - a0);
            const int nb = max(0, min(run, L - a0 - na));
            const uint64_t* A = src + a0;
            const uint64_t* Bv = src + a0 + na;
            const int total = na + nb;
            const int per = (total + blockDim.x - 1) / blockDim.x;
            const int k0 = min(total, (int)threadIdx.x * per), k1 = min(total, k0 + per);
            if (k0 < k1) {
                // merge path: i elements from A and k0 - i from B precede output k0
                int lo = max(0, k0 - nb), hi = min(k0, na);
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (A[mid] < Bv[k0 - mid - 1]) lo = mid + 1;
                    else hi = mid;
                }
                int i = lo, j = k0 - lo;
                for (int k = k0; k < k1; ++k) {
                    const bool takeA = j >= nb || (i < na && A[i] < Bv[j]);
                    dst[a0 + k] = takeA ? A[i++] : Bv[j++];
                }
            }
        }
        __syncthreads();
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    *result = src;
}

__global__ void __launch_bounds__(TS_THREADS) tile_sort_kernel(const uint32_t* __restrict__ tile_start,
                                                               const uint32_t* __restrict__ tile_cnt, int T,
                                                               int64_t cap, uint64_t* __restrict__ bucket,
                                                               uint64_t* __restrict__ tmp, uint32_t* __restrict__ gids,
                                                               uint2* __restrict__ ranges) {
    __shared__ uint64_t s[TS_CAP];
    const int t = blockIdx.x;
    if (t >= T) return;
    const int64_t start = tile_start[t];
    int64_t end = start + tile_cnt[t];
    if (end > cap) end = cap;                 // capacity overflow: keep every access in bounds
    const int L = end > start ? (int)(end - start) : 0;
    const uint32_t s0 = (uint32_t)(start < cap ? start : cap);   // [s0, s0 + L) lies within capacity
    if (threadIdx.x == 0) ranges[t] = make_uint2(s0, s0 + (uint32_t)L);
    if (L == 0) return;
    uint64_t* res = nullptr;
    sort_segment(bucket + start, tmp + start, L, s, &res);
    for (int k = threadIdx.x; k < L; k += blockDim.x) gids[start + k] = (uint32_t)(res[k] & 0xffffffffu);
}

__global__ void keys_kernel(const uint2* __restrict__ ranges, int T, const uint32_t* __restrict__ gids,
                            const float* __restrict__ depth, uint64_t* __restrict__ keys) {
    const int t = blockIdx.x;
    if (t >= T) return;
    const uint2 r = ranges[t];
    for (uint32_t k = r.x + threadIdx.x; k < r.y; k += blockDim.x)
        keys[k] = ((uint64_t)(uint32_t)t << 32) | (uint64_t)__float_as_uint(depth[gids[k]]);
}

struct BinWs {
    uint32_t *cnt_pad, *fill_pad, *tile_cnt, *tile_start;
    uint64_t *bucket, *tmp;
    void* scan_tmp;
    size_t bytes;
};

static BinWs carve_bin_ws(void* base, int64_t cap, int T) {
    Carver c{reinterpret_cast<char*>(base), 0};
    BinWs w;
    const size_t tt = (size_t)(T > 0 ? T : 1);
    const size_t cc = (size_t)(cap > 0 ? cap : 1);
    w.cnt_pad = c.take<uint32_t>(2 * tt * kPad);   // counts and fill cursors, zeroed together
    w.fill_pad = w.cnt_pad + tt * kPad;
    w.tile_cnt = c.take<uint32_t>(tt);
    w.tile_start = c.take<uint32_t>(tt);
    w.bucket = c.take<uint64_t>(cc);
    w.tmp = c.take<uint64_t>(cc);
    w.scan_tmp = c.take<char>(scan_tmp_bytes(T));
    w.bytes = c.off + 256;
    return w;
}

size_t bin_sort_ws_bytes(int n, int64_t capacity, int num_tiles) {
    (void)n;
    return carve_bin_ws(nullptr, capacity, num_tiles).bytes;
}

cudaError_t launch_bin_sort(const sgs_proj& proj, const ViewsDev& vd, const SetDev& st, const sgs_bins& out, void* ws,
                            cudaStream_t stream) {
    (void)st;
    const int n = vd.row_off[vd.nv];            // projection rows
    const int T = vd.T_total;
    BinWs w = carve_bin_ws(ws, out.capacity, T);
    cudaError_t e = cudaMemsetAsync(w.cnt_pad, 0, 2 * sizeof(uint32_t) * kPad * (size_t)T, stream);
    if (e != cudaSuccess) return e;
    const int nb = (n + 255) / 256;
    const short4* rect = reinterpret_cast<const short4*>(proj.rect);
    if (n > 0) {
        tile_count_kernel<<<nb, 256, 0, stream>>>(rect, proj.tiles_touched, n, vd, w.cnt_pad);
        note_launch();
    }
    unpad_kernel<<<(T + 255) / 256, 256, 0, stream>>>(w.cnt_pad, T, w.tile_cnt);
    note_launch();
    // per-tile ranges: exclusive scan of the counts; the total is M
    e = launch_exclusive_scan(w.tile_cnt, w.tile_start, reinterpret_cast<uint32_t*>(out.count), T, nullptr,
                              w.scan_tmp, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        emit_kernel<<<nb, 256, 0, stream>>>(rect, proj.tiles_touched, proj.depth, n, vd, w.tile_start, w.fill_pad,
                                            out.capacity, w.bucket);
        note_launch();
    }
    tile_sort_kernel<<<T, TS_THREADS, 0, stream>>>(w.tile_start, w.tile_cnt, T, out.capacity, w.bucket, w.tmp,
                                                   out.gids, reinterpret_cast<uint2*>(out.ranges));
    note_launch();
    if (out.keys) {
        keys_kernel<<<T, 128, 0, stream>>>(reinterpret_cast<const uint2*>(out.ranges), T, out.gids, proj.depth,
                                            out.keys);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace sgs
