// spl_sort.cu -- depth ordering of the tile lists for the general absorption
// form (Eq. 1 with E_p != A_p), where the particles a ray crosses must be
// taken in depth order (the sort step of Sec. 4 with a depth key).
//
// A stable least-significant-digit radix sort of 64-bit keys, 8-bit digits:
// per pass, every block of kSortTile keys counts its digits (hist[digit][block]),
// one exclusive scan over the digit-major table gives every (digit, block) its
// output base, and every block scatters its keys in their original order.
// Stability inside a block: each warp owns a contiguous run of keys taken 32
// at a time; lanes holding the same digit are ranked with a match mask, the
// warp keeps a running count per digit, and the warps' per-digit counts are
// prefixed in shared memory.
//
// Depth order of a frame (spl_api.cu): (1) particles by (depth key, index) --
// key = (float bits of z_c) << 32 | index, inactive and non-absorbing
// particles last -- which gives every particle its rank; (2) the entries of
// the tile lists by (tile, rank), which keeps every tile's range in place and
// orders it front to back.
#include "spl_geom.cuh"

namespace spl {

constexpr int kSortThreads = 256;
// keys per thread: 8 keep the scatter at 48 registers and 5 CTAs per SM
// without spills (16 took 99 registers, 2 CTAs per SM; the scatter and depth
// sort of the clustered 10M frame went from 4.64 to 3.77 ms, same result; 4
// keys per thread at 6 or 8 CTAs per SM: 4.12 and 3.84 ms)
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;            // keys per block

__device__ __forceinline__ unsigned digit_of(unsigned long long k, int shift) {
    return (unsigned)(k >> shift) & 0xFFu;
}

// hist[d * nblocks + b] = keys of block b with digit d.
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const unsigned long long *keys,
                                                                  int64_t n, int shift, int *hist,
                                                                  int nblocks) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const int64_t i = b0 + k;
        if (i < n) atomicAdd(&cnt[digit_of(keys[i], shift)], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of block b's keys to base[d * nblocks + b] + rank.
__global__ void __launch_bounds__(kSortThreads, 5) radix_scatter_kernel(const unsigned long long *in,
                                                                     unsigned long long *out,
                                                                     int64_t n, int shift,
                                                                     const int *base, int nblocks) {
    constexpr int NW = kSortThreads / 32;
    __shared__ int wcnt[NW][256];      // per warp and digit: count, then offset
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    // warp w owns keys [b0 + w * 32 * kSortItems, ... + 32 * kSortItems), in
    // rounds of 32 consecutive keys
    const int64_t w0 = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kSortItems;
    unsigned long long key[kSortItems];
    int rnk[kSortItems];
    // all of the warp's keys are loaded before the ranking rounds, whose warp
    // barriers would otherwise serialise the loads' latencies
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = w0 + r * 32 + lane;
        key[r] = i < n ? in[i] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = w0 + r * 32 + lane;
        const bool valid = i < n;
        const int d = valid ? (int)digit_of(key[r], shift) : -1;
        const unsigned m = __match_any_sync(0xffffffffu, d);
        int before = 0;
        if (valid) before = wcnt[warp][d];
        rnk[r] = before + __popc(m & lt);
        __syncwarp();
        if (valid && lane == __ffs(m) - 1) wcnt[warp][d] = before + __popc(m);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps inside the block, plus the block's base
    {
        const int d = threadIdx.x;     // kSortThreads == 256 digits
        int run = base[d * nblocks + blockIdx.x];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = w0 + r * 32 + lane;
        if (i < n) out[wcnt[warp][digit_of(key[r], shift)] + rnk[r]] = key[r];
    }
}

int radix_blocks(int64_t n) { return (int)((n + kSortTile - 1) / kSortTile); }

// Exclusive scan of m ints for the digit table: blocks of kScanChunk values
// are reduced, the block sums scanned by one CTA (scan_kernel), and every
// block then scans its values from its base.  out[m] = total.
constexpr int kScanThreads = 1024, kScanPer = 8, kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive(int v, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    total = wsum[32];
    const int r = wsum[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int *in, int m, int *part) {
    __shared__ int wsum[33];
    const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int v = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < m) v += in[base + k];
    int total;
    block_exclusive(v, wsum, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int *in, int m,
                                                                  const int *pbase, int nparts,
                                                                  int *out) {
    __shared__ int wsum[33];
    const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int v[kScanPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < m ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = pbase[blockIdx.x] + block_exclusive(sum, wsum, total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < m) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = pbase[nparts];
}

static int scan_parts(int m) { return (m + kScanChunk - 1) / kScanChunk; }

// Ints of radix scratch for n keys: digit counts, scanned bases, block sums.
int64_t radix_scratch_ints(int64_t n) {
    const int64_t nb = radix_blocks(n > 0 ? n : 1);
    const int64_t parts = scan_parts((int)(256 * nb));
    return 512 * nb + 2 + 2 * (parts + 1);
}

static void scan_digits(int m, const int *in, int *out, int *part, int *pbase, cudaStream_t s) {
    const int np = scan_parts(m);
    scan_reduce_kernel<<<np, kScanThreads, 0, s>>>(in, m, part);
    ++g_launches;
    launch_scan(np, part, pbase, nullptr, 0, nullptr, s);
    scan_apply_kernel<<<np, kScanThreads, 0, s>>>(in, m, pbase, np, out);
    ++g_launches;
}

// Sorts keys[0, n) by the 8-bit digits at the given shifts (least
// significant first); tmp holds n keys; hist holds radix_scratch_ints(n)
// ints.  Returns the array holding the result (keys or tmp).
unsigned long long *launch_radix_sort(unsigned long long *keys, unsigned long long *tmp, int64_t n,
                                      const int *shifts, int npasses, int *hist, cudaStream_t s) {
    if (n <= 0) return keys;
    const int nb = radix_blocks(n);
    const int m = 256 * nb, np = scan_parts(m);
    int *cnt = hist, *bases = hist + m + 1, *part = bases + m + 1, *pbase = part + np + 1;
    unsigned long long *a = keys, *b = tmp;
    for (int p = 0; p < npasses; ++p) {
        radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(a, n, shifts[p], cnt, nb);
        ++g_launches;
        scan_digits(m, cnt, bases, part, pbase, s);
        radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(a, b, n, shifts[p], bases, nb);
        ++g_launches;
        unsigned long long *t = a;
        a = b;
        b = t;
    }
    return a;
}

// ---------------------------------------------------------------------------
// Depth order of a frame.
// ---------------------------------------------------------------------------

// Particle keys: (float bits of the depth key) << 32 | index; the depth key is
// positive for every active particle (z_c > z_near > 0), so its bits order as
// the value.  Inactive or non-absorbing records go last.
__global__ void depth_keys_kernel(const Rec *recs, const float2 *rec2, int64_t n,
                                  unsigned long long *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 q = rec2[i];
        const bool live = recs[i].r1.x >= 0.f && q.x > 0.f;
        const unsigned hi = live ? __float_as_uint(q.y) : 0xFFFFFFFFu;
        keys[i] = ((unsigned long long)hi << 32) | (unsigned long long)(unsigned)i;
    }
}

// rank[id] = position of particle id in the sorted order.
__global__ void rank_kernel(const unsigned long long *sorted, int64_t n, unsigned *rank) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        rank[(unsigned)(sorted[k] & 0xFFFFFFFFull)] = (unsigned)k;
}

// Entry keys of the list region [e0, e1): (tile << 32) | rank[entry], the tile
// found by bisection of the region's slot offsets off[0 .. ntiles].
__global__ void entry_keys_kernel(const unsigned *entries, const long long *off, int ntiles,
                                  const unsigned *rank, unsigned long long *keys) {
    const long long e0 = off[0], e1 = off[ntiles];
    for (long long k = e0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < e1;
         k += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = ntiles - 1;          // last tile with off[t] <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        keys[k - e0] = ((unsigned long long)(unsigned)lo << 32) | rank[entries[k]];
    }
}

// entries[off[0] + k] = the particle of rank (keys[k] & mask): the index of
// rank r is the low half of the r-th sorted particle key.
__global__ void entry_store_kernel(const unsigned long long *keys, const long long *off, int ntiles,
                                   const unsigned long long *sorted_particles, unsigned *entries) {
    const long long e0 = off[0], count = off[ntiles] - e0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned r = (unsigned)(keys[k] & 0xFFFFFFFFull);
        entries[e0 + k] = (unsigned)(sorted_particles[r] & 0xFFFFFFFFull);
    }
}

static int bits_for(unsigned long long v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0ull) ++b;
    return b;
}

// Whole depth ordering for one view whose entries all sit in the medium list
// slots off[0 .. ntiles] (device offsets into entries; the host passes their
// total, off[ntiles] - off[0], known after the binning synchronisation).
// pkeys/ptmp: n particle keys each; ekeys/etmp: total entry keys each;
// rank: n; hist: radix_scratch_ints(max(n, total)) ints.
void launch_depth_order(const Rec *recs, const float2 *rec2, int64_t n, unsigned *entries,
                        const long long *off, int ntiles, long long total, unsigned long long *pkeys,
                        unsigned long long *ptmp, unsigned long long *ekeys,
                        unsigned long long *etmp, unsigned *rank, int *hist, int sms,
                        cudaStream_t s) {
    if (n <= 0 || total <= 0) return;
    depth_keys_kernel<<<sms * 8, 256, 0, s>>>(recs, rec2, n, pkeys);
    ++g_launches;
    int shifts[8], np = 0;
    const int idb = bits_for((unsigned long long)(n - 1));
    // the keys start in index order and every pass is stable, so sorting by
    // the depth bits alone leaves equal depths in index order: the index bits
    // need no passes of their own
    for (int sh = 32; sh < 64; sh += 8) shifts[np++] = sh;
    unsigned long long *ps = launch_radix_sort(pkeys, ptmp, n, shifts, np, hist, s);
    rank_kernel<<<sms * 8, 256, 0, s>>>(ps, n, rank);
    ++g_launches;
    entry_keys_kernel<<<sms * 8, 256, 0, s>>>(entries, off, ntiles, rank, ekeys);
    ++g_launches;
    np = 0;
    for (int sh = 0; sh < idb; sh += 8) shifts[np++] = sh;
    const int tb = bits_for((unsigned long long)(ntiles - 1));
    for (int sh = 32; sh < 32 + tb; sh += 8) shifts[np++] = sh;
    unsigned long long *es = launch_radix_sort(ekeys, etmp, total, shifts, np, hist, s);
    entry_store_kernel<<<sms * 8, 256, 0, s>>>(es, off, ntiles, ps, entries);
    ++g_launches;
}

}  // namespace spl
