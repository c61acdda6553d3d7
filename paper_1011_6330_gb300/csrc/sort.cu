// Stable re-sort of a tube's particle slots by position: an LSD radix sort of
// (position key, slot) pairs with 8-bit digits, the key being the position on
// a grid of 256 bins per cell (fewer on grids of more than 2^23 cells), then a
// gather of positions, momenta and IDs. Holes sort last and drop out.
//
// The physics does not depend on the slot order (the current and the base
// weight are exact integer sums); the sort restores the cell locality that
// the particle kernel's per-thread runs rely on, and groups the particles that
// are about to cross a node so that few warps take the rare branch.
#include "device_common.cuh"

namespace sclf {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                          // per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // items per tile
constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;

// Key of slot i: its position on a grid of 2^sub bins per cell, floor(x 2^sub)
// (so that particles about to cross a node end up next to each other), or
// nz 2^sub for a hole. scale converts a stored position to cells.
template <class Pos>
__global__ void sort_keys_kernel(const Pos* xi, long long n, int nz, double scale, int sub,
                                 unsigned* keys, unsigned* vals) {
    const unsigned top = static_cast<unsigned>(nz) << sub;
    const double sc = ldexp(scale, sub);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const Pos x = xi[i];
        unsigned k = top;
        if (x >= Pos(0)) {
            const double c = floor(static_cast<double>(x) * sc);
            k = c < double(top) ? static_cast<unsigned>(c) : top;
        }
        keys[i] = k;
        vals[i] = static_cast<unsigned>(i);
    }
}

// Per tile: histogram of the pass's digit; hist is digit-major
// (hist[d * ntiles + tile]) so that its exclusive scan is each (digit, tile)'s
// first output position.
__global__ void __launch_bounds__(kSortThreads)
sort_hist_kernel(const unsigned* keys, long long n, int shift, long long ntiles,
                 unsigned* hist) {
    __shared__ unsigned h[kRadix];
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) h[d] = 0;
        __syncthreads();
        const long long base = tile * kSortTile;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const long long i = base + k * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d * ntiles + tile] = h[d];
        __syncthreads();
    }
}

// Exclusive scan of m unsigned values in place, in three launches: block
// sums, a single-block scan of them, and the block-local scans plus offsets.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* sh, unsigned* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned o = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += o;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned y = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned o = __shfl_up_sync(kFull, y, off);
            if (lane >= off) y += o;
        }
        if (lane < nw) sh[lane] = y;
    }
    __syncthreads();
    const unsigned wbase = w > 0 ? sh[w - 1] : 0u;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wbase + x - v;
}

__global__ void __launch_bounds__(kScanBlock) scan_partials_kernel(const unsigned* a, long long m,
                                                                   unsigned* partial) {
    __shared__ unsigned sh[32];
    const long long i = blockIdx.x * static_cast<long long>(kScanBlock) + threadIdx.x;
    unsigned total;
    block_excl_scan(i < m ? a[i] : 0u, sh, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) scan_partial_sums_kernel(unsigned* partial,
                                                                       long long nb) {
    __shared__ unsigned sh[32];
    unsigned carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += kScanBlock) {
        const long long i = b0 + threadIdx.x;
        const unsigned v = i < nb ? partial[i] : 0u;
        unsigned total;
        const unsigned ex = block_excl_scan(v, sh, &total);
        if (i < nb) partial[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_finish_kernel(unsigned* a, long long m,
                                                                 const unsigned* partial) {
    __shared__ unsigned sh[32];
    const long long i = blockIdx.x * static_cast<long long>(kScanBlock) + threadIdx.x;
    unsigned total;
    const unsigned ex = block_excl_scan(i < m ? a[i] : 0u, sh, &total);
    if (i < m) a[i] = partial[blockIdx.x] + ex;
}

// Per tile: each item's rank among the tile's items with the same digit that
// come before it, then the scatter to offset(digit, tile) + rank. Items are
// visited in index order: round r holds items [r * 256, r * 256 + 256) of the
// tile, one per thread in thread order; inside a warp the rank comes from
// the lanes with the same digit (match), across the warps of a round from
// per-warp digit counts in shared memory, across rounds from a running count.
__global__ void __launch_bounds__(kSortThreads)
sort_scatter_kernel(const unsigned* keys, const unsigned* vals, long long n, int shift,
                    long long ntiles, const unsigned* offs, unsigned* keys_out,
                    unsigned* vals_out) {
    __shared__ unsigned running[kRadix];
    __shared__ unsigned wcount[kWarps][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) running[d] = 0;
        const long long base = tile * kSortTile;
        for (int r = 0; r < kSortItems; ++r) {
            for (int d = threadIdx.x; d < kRadix * kWarps; d += kSortThreads)
                (&wcount[0][0])[d] = 0;
            __syncthreads();
            const long long i = base + r * kSortThreads + threadIdx.x;
            const bool valid = i < n;
            const unsigned key = valid ? keys[i] : 0u;
            const unsigned val = valid ? vals[i] : 0u;
            const unsigned d = (key >> shift) & (kRadix - 1);
            // lanes of this warp with the same digit (invalid lanes use a digit
            // of their own that no valid lane has: kRadix + lane)
            const unsigned tag = valid ? d : static_cast<unsigned>(kRadix + lane);
            const unsigned peers = __match_any_sync(kFull, tag);
            const unsigned in_warp = __popc(peers & lt_mask);
            const bool leader = (peers & lt_mask) == 0u;
            if (valid && leader) wcount[w][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                unsigned before = running[d];
                for (int ww = 0; ww < w; ++ww) before += wcount[ww][d];
                const unsigned dst = offs[static_cast<long long>(d) * ntiles + tile] + before +
                                     in_warp;
                keys_out[dst] = key;
                vals_out[dst] = val;
            }
            __syncthreads();
            for (int dd = threadIdx.x; dd < kRadix; dd += kSortThreads) {
                unsigned add = 0;
                for (int ww = 0; ww < kWarps; ++ww) add += wcount[ww][dd];
                running[dd] += add;
            }
            __syncthreads();
        }
    }
}

// Slots [0, n_live) <- the sorted slots: out[i] = in[perm[i]].
template <class Pos, class Mom>
__global__ void sort_gather_kernel(const unsigned* perm, long long n_live, const Pos* xi,
                                   const Mom* u, const long long* ids, Pos* xo, Mom* uo,
                                   long long* io) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
         i < n_live; i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned j = perm[i];
        xo[i] = xi[j];
        uo[i] = u[j];
        if (ids) io[i] = ids[j];
    }
}

int grid_of(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return static_cast<int>(g < cap ? g : cap);
}

}  // namespace

// Scratch the sort needs for n slots (bytes).
long long sort_scratch_bytes(long long n) {
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long m = kRadix * ntiles;
    const long long nb = (m + kScanBlock - 1) / kScanBlock;
    auto al = [](long long b) { return (b + 255) / 256 * 256; };
    return 4 * al(4 * n) + al(4 * m) + al(4 * nb);
}

template <class Pos, class Mom>
cudaError_t launch_sort_by_cell(const Pos* xi, const Mom* u, const long long* ids, long long n,
                                int nz, double scale, void* scratch, Pos* xo, Mom* uo,
                                long long* io, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long m = kRadix * ntiles;
    const long long nb = (m + kScanBlock - 1) / kScanBlock;
    auto al = [](long long b) { return (b + 255) / 256 * 256; };
    char* p = static_cast<char*>(scratch);
    unsigned* keys[2] = {reinterpret_cast<unsigned*>(p), reinterpret_cast<unsigned*>(p + al(4 * n))};
    unsigned* vals[2] = {reinterpret_cast<unsigned*>(p + 2 * al(4 * n)),
                         reinterpret_cast<unsigned*>(p + 3 * al(4 * n))};
    unsigned* hist = reinterpret_cast<unsigned*>(p + 4 * al(4 * n));
    unsigned* partial = reinterpret_cast<unsigned*>(p + 4 * al(4 * n) + al(4 * m));

    // sub-cell bits: up to 8, keeping the hole key nz 2^sub below 2^31
    int cbits = 0;
    while ((1LL << cbits) <= nz) ++cbits;
    const int sub = cbits + 8 <= 31 ? 8 : 31 - cbits;
    sort_keys_kernel<Pos><<<grid_of(n, 256, 8192), 256, 0, s>>>(xi, n, nz, scale, sub, keys[0],
                                                               vals[0]);
    const int bits = cbits + sub;                        // keys are 0..nz 2^sub
    const int tiles_grid = static_cast<int>(ntiles < 65535 * 8 ? ntiles : 65535 * 8);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        sort_hist_kernel<<<tiles_grid, kSortThreads, 0, s>>>(keys[cur], n, shift, ntiles, hist);
        scan_partials_kernel<<<static_cast<int>(nb), kScanBlock, 0, s>>>(hist, m, partial);
        scan_partial_sums_kernel<<<1, kScanBlock, 0, s>>>(partial, nb);
        scan_finish_kernel<<<static_cast<int>(nb), kScanBlock, 0, s>>>(hist, m, partial);
        sort_scatter_kernel<<<tiles_grid, kSortThreads, 0, s>>>(
            keys[cur], vals[cur], n, shift, ntiles, hist, keys[cur ^ 1], vals[cur ^ 1]);
        cur ^= 1;
    }
    // the gather covers all n slots, holes last; the caller keeps the live
    // ones (n minus the holes, from the device counters)
    sort_gather_kernel<Pos, Mom><<<grid_of(n, 256, 8192), 256, 0, s>>>(vals[cur], n, xi, u, ids,
                                                                      xo, uo, io);
    return cudaGetLastError();
}

template cudaError_t launch_sort_by_cell<float, float>(const float*, const float*,
                                                       const long long*, long long, int, double,
                                                       void*, float*, float*, long long*,
                                                       cudaStream_t);
template cudaError_t launch_sort_by_cell<double, double>(const double*, const double*,
                                                         const long long*, long long, int, double,
                                                         void*, double*, double*, long long*,
                                                         cudaStream_t);
template cudaError_t launch_sort_by_cell<int, float>(const int*, const float*, const long long*,
                                                     long long, int, double, void*, int*, float*,
                                                     long long*, cudaStream_t);

}  // namespace sclf
