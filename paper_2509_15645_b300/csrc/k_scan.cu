// k_scan.cu -- device-wide exclusive scan and ordered compaction of a
// bitmask, with data-dependent lengths read from device memory so that callers
// never synchronise (graph capture).
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;

__device__ __forceinline__ int scan_length(ScanLen L)
{
    if (!L.n_dev) return L.fixed;
    int n = *L.n_dev;
    if (L.cap > 0 && n > L.cap) n = L.cap;
    return L.mul * ((n + L.div - 1) / L.div) + L.add;
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *total, uint32_t *s_warp)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    uint32_t r = s_warp[wid] + incl - x;
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, ScanLen L, uint32_t *partials)
{
    __shared__ uint32_t s_warp[33];
    int len = scan_length(L);
    int seg = (len + gridDim.x - 1) / gridDim.x;
    int lo = blockIdx.x * seg, hi = min(len, lo + seg);
    uint32_t acc = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += in[i];
    uint32_t tot;
    block_excl_scan(acc, &tot, s_warp);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void k_scan_partials(uint32_t *partials, int g, int *total_out, int total_cap, int *status)
{
    __shared__ uint32_t s_warp[33];
    // g <= 1024: each of 256 threads holds up to 4 partials
    uint32_t v[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        int idx = threadIdx.x * 4 + j;
        v[j] = idx < g ? partials[idx] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(s, &tot, s_warp);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        int idx = threadIdx.x * 4 + j;
        if (idx < g) partials[idx] = ex;
        ex += v[j];
    }
    if (threadIdx.x == 0 && total_out) {
        // compared unsigned: a total past 2^31 (only from counts that are not
        // a cull's) must not pass as a negative count
        uint32_t t = tot;
        if (total_cap > 0 && t > (uint32_t)total_cap) {
            if (status) latch(status, GS_ERR_CAPACITY);
            t = (uint32_t)total_cap;
        }
        *total_out = (int)min(t, 0x7fffffffu);
    }
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, ScanLen L, const uint32_t *__restrict__ partials)
{
    __shared__ uint32_t s_warp[33];
    int len = scan_length(L);
    int seg = (len + gridDim.x - 1) / gridDim.x;
    int lo = blockIdx.x * seg, hi = min(len, lo + seg);
    uint32_t carry = partials[blockIdx.x];
    for (int base = lo; base < hi; base += SCAN_BLOCK * SCAN_ITEMS) {
        uint32_t v[SCAN_ITEMS], s = 0;
        int i0 = base + threadIdx.x * SCAN_ITEMS;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            v[j] = (i0 + j < hi) ? in[i0 + j] : 0u;
            s += v[j];
        }
        uint32_t tot;
        uint32_t ex = block_excl_scan(s, &tot, s_warp) + carry;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            if (i0 + j < hi) out[i0 + j] = ex;
            ex += v[j];
        }
        carry += tot;
    }
}

void scan_exclusive(const uint32_t *in, uint32_t *out, ScanLen L, Work &w, int *total_out, int total_cap,
                    cudaStream_t s)
{
    int g = w.scan_grid;
    k_scan_reduce<<<g, SCAN_BLOCK, 0, s>>>(in, L, w.partials);
    k_scan_partials<<<1, 256, 0, s>>>(w.partials, g, total_out, total_cap, w.status);
    k_scan_down<<<g, SCAN_BLOCK, 0, s>>>(in, out, L, w.partials);
}

// ---------------------------------------------------------------------------
// Exclusive scan of up to SMALL_SCAN_MAX chunk counts in place, by one block
// (one launch instead of the three of scan_exclusive): each thread scans a
// contiguous segment, the block scans the segment sums.  Writes the total to
// total_out (clamped to total_cap, GS_ERR_CAPACITY latched above it).
constexpr int SMALL_SCAN_THREADS = 1024;
constexpr int64_t SMALL_SCAN_MAX = 8 * SMALL_SCAN_THREADS;   // longer scans: three kernels (the one-block scan walks its segments serially)

__global__ void __launch_bounds__(SMALL_SCAN_THREADS) k_scan_small(uint32_t *v, int len, int *total_out,
                                                                   int total_cap, int *status)
{
    __shared__ uint32_t s_warp[33];
    const int seg = (len + SMALL_SCAN_THREADS - 1) / SMALL_SCAN_THREADS;
    const int lo = threadIdx.x * seg, hi = min(len, lo + seg);
    uint32_t sum = 0;
    for (int k = lo; k < hi; k++) sum += v[k];
    uint32_t tot;
    uint32_t ex = block_excl_scan(sum, &tot, s_warp);
    for (int k = lo; k < hi; k++) {
        const uint32_t x = v[k];
        v[k] = ex;
        ex += x;
    }
    if (threadIdx.x == 0 && total_out) {
        // compared unsigned: a total past 2^31 (only from counts that are not
        // a cull's) must not pass as a negative count
        uint32_t t = tot;
        if (total_cap > 0 && t > (uint32_t)total_cap) {
            if (status) latch(status, GS_ERR_CAPACITY);
            t = (uint32_t)total_cap;
        }
        *total_out = (int)min(t, 0x7fffffffu);
    }
}

void scan_counts(uint32_t *v, int64_t len, int *total_out, int cap, Work &w, cudaStream_t s)
{
    if (len <= SMALL_SCAN_MAX) {
        k_scan_small<<<1, SMALL_SCAN_THREADS, 0, s>>>(v, (int)len, total_out, cap, w.status);
    } else {
        ScanLen L{nullptr, 1, 1, 0, (int)len, 0};
        scan_exclusive(v, v, L, w, total_out, cap, s);
    }
}

// Ordered compaction of a bitmask (bit i of word i/32), one 256-thread block
// per chunk of CHUNK_WORDS words at a time; warp k takes words k, k + 8, ...
// and a lane the bit of its index.  chunk_ofs holds the exclusive scan of
// per-chunk popcounts.  Writes ids (ascending, only those below cap) and
// word_prefix[w] = number of set bits before word w.  A warp issues all its
// mask words and (for the optimizer's update set) all its members' counter
// reads before the first store, so a chunk costs one memory latency.
constexpr int COMPACT_BLOCK = 256, COMPACT_WPW = CHUNK_WORDS / (COMPACT_BLOCK / 32);

__global__ void __launch_bounds__(COMPACT_BLOCK) k_compact_mask(const uint32_t *__restrict__ mask, int64_t n,
                                                                int64_t nwords,
                                                                const uint32_t *__restrict__ chunk_ofs, int32_t *ids,
                                                                uint32_t *word_prefix, int cap, uint8_t *counter,
                                                                uint8_t *delay)
{
    __shared__ uint32_t s_pref[CHUNK_WORDS];
    __shared__ uint32_t s_warp[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nchunks = (nwords + CHUNK_WORDS - 1) / CHUNK_WORDS;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t w0 = c * CHUNK_WORDS;
        uint32_t mw[COMPACT_WPW];
#pragma unroll
        for (int k = 0; k < COMPACT_WPW; k++) {
            const int64_t wd = w0 + wid + k * (COMPACT_BLOCK / 32);
            mw[k] = wd < nwords ? __ldg(mask + wd) : 0u;
        }
        uint8_t cv[COMPACT_WPW];
        if (counter) {
#pragma unroll
            for (int k = 0; k < COMPACT_WPW; k++) {
                const int64_t id = (w0 + wid + k * (COMPACT_BLOCK / 32)) * 32 + lane;
                cv[k] = ((mw[k] >> lane) & 1u) ? counter[id] : (uint8_t)0;
            }
        }
        uint32_t word = 0;
        if (threadIdx.x < CHUNK_WORDS && w0 + threadIdx.x < nwords) word = __ldg(mask + w0 + threadIdx.x);
        const uint32_t cnt = threadIdx.x < CHUNK_WORDS ? __popc(word) : 0u;
        const uint32_t ex = block_excl_scan(cnt, nullptr, s_warp);
        const uint32_t base = __ldg(chunk_ofs + c);
        if (threadIdx.x < CHUNK_WORDS) {
            s_pref[threadIdx.x] = base + ex;
            if (w0 + threadIdx.x < nwords && word_prefix) word_prefix[w0 + threadIdx.x] = base + ex;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < COMPACT_WPW; k++) {
            const int j = wid + k * (COMPACT_BLOCK / 32);
            const uint32_t m = mw[k];
            if ((m >> lane) & 1u) {
                const uint32_t pos = s_pref[j] + __popc(m & ((1u << lane) - 1u));
                const int64_t id = (w0 + j) * 32 + lane;
                if (pos < (uint32_t)cap && id < n) {     // unsigned: no offset passes as negative
                    if (ids) ids[pos] = (int32_t)id;
                    if (counter) {           // optimizer update set: record the delay, clear the counter
                        delay[pos] = cv[k];
                        counter[id] = 0;
                    }
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_chunk_counts(const uint32_t *__restrict__ mask, int64_t nwords, uint32_t *chunk_cnt)
{
    int64_t nchunks = (nwords + CHUNK_WORDS - 1) / CHUNK_WORDS;
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        int64_t w0 = c * CHUNK_WORDS;
        uint32_t s = 0;
        for (int j = lane; j < CHUNK_WORDS; j += 32)
            if (w0 + j < nwords) s += __popc(mask[w0 + j]);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) chunk_cnt[c] = s;
    }
}

void compact_mask(const uint32_t *mask, int64_t n, uint32_t *chunk_cnt, bool have_counts, int32_t *ids,
                  uint32_t *word_prefix, int cap, int *count_out, Work &w, cudaStream_t s, uint8_t *counter,
                  uint8_t *delay)
{
    int64_t nwords = (n + 31) / 32;
    int64_t nchunks = (nwords + CHUNK_WORDS - 1) / CHUNK_WORDS;
    if (!have_counts)
        k_chunk_counts<<<w.grid(nchunks * 32, 256), 256, 0, s>>>(mask, nwords, chunk_cnt);
    scan_counts(chunk_cnt, nchunks, count_out, cap, w, s);
    k_compact_mask<<<w.grid(nchunks * COMPACT_BLOCK, COMPACT_BLOCK), COMPACT_BLOCK, 0, s>>>(
        mask, n, nwords, chunk_cnt, ids, word_prefix, cap, counter, delay);
}

// dst[k] = src[ids[k]] for k < min(*n, cap): a byte per id (defer counters of
// a compact id list).
__global__ void k_gather_u8(const uint8_t *__restrict__ src, const int32_t *__restrict__ ids, const int *n_p, int cap,
                            uint8_t *__restrict__ dst)
{
    const int n = min(*n_p, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[k] = src[ids[k]];
}

// dst[k * planes + r] = src[r * spitch + k] for k < min(*n, cap), r < planes:
// plane-major rows to one row per element, through 32 x 32 shared tiles so
// both sides are coalesced.
__global__ void k_to_rows(const float *__restrict__ src, int64_t spitch, int planes, const int *n_p, int cap,
                          float *__restrict__ dst)
{
    __shared__ float tile[32][33];
    const int n = min(*n_p, cap);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8 threads
    const int rt = (planes + 31) / 32;
    for (int64_t b = blockIdx.x; b < (int64_t)rt * ((n + 31) / 32); b += gridDim.x) {
        const int r0 = (int)(b % rt) * 32;
        const int64_t k0 = (b / rt) * 32;
        for (int j = ty; j < 32; j += 8)
            if (r0 + j < planes && k0 + tx < n) tile[j][tx] = src[(int64_t)(r0 + j) * spitch + k0 + tx];
        __syncthreads();
        for (int j = ty; j < 32; j += 8)
            if (k0 + j < n && r0 + tx < planes) dst[(k0 + j) * planes + r0 + tx] = tile[tx][j];
        __syncthreads();
    }
}

void launch_to_rows(const float *src, int64_t spitch, int planes, const int *n, int cap, float *dst, Work &w,
                    cudaStream_t s)
{
    const int64_t tiles = (int64_t)((planes + 31) / 32) * ((cap + 31) / 32);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(tiles, 1), (int64_t)w.num_sms * 16);
    k_to_rows<<<grid, 256, 0, s>>>(src, spitch, planes, n, cap, dst);
}

void launch_gather_u8(const uint8_t *src, const int32_t *ids, const int *n, int cap, uint8_t *dst, Work &w,
                      cudaStream_t s)
{
    k_gather_u8<<<w.grid(cap, 256, 4), 256, 0, s>>>(src, ids, n, cap, dst);
}

}  // namespace gs
