// Stable in-place removal of the holes that removed particles leave in the
// slot arrays (single pass, decoupled look-back).
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// In-place stable compaction (decoupled look-back)
// ---------------------------------------------------------------------------
constexpr unsigned kFlagAgg = 1u, kFlagIncl = 2u;

__device__ __forceinline__ unsigned long long pack_state(unsigned epoch, unsigned flag,
                                                         unsigned value) {
    return (static_cast<unsigned long long>(epoch & 0x3fffffffu) << 34) |
           (static_cast<unsigned long long>(flag) << 32) | value;
}
__device__ __forceinline__ void store_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <class Pos, class Mom>
__global__ void __launch_bounds__(kThreads) compact_kernel(const CompactArgs<Pos, Mom> a) {
    using L = Layout<Pos>;
    static_assert(Layout<Pos>::kPPT == Layout<Mom>::kPPT, "one tile shape");
    constexpr int kPPT = L::kPPT, kVec = L::kVec, kTile = L::kTile;
    __shared__ long long s_tile;
    __shared__ int s_warp[kThreads / 32];
    __shared__ long long s_prefix;

    DevState* st = a.st;
    const long long n_slots = st->n_slots;
    const unsigned epoch = st->compact_epoch;
    const long long ntiles = (n_slots + kTile - 1) / kTile;
    // Holes cost one 8-byte read per step each; moving every slot behind the
    // first hole costs 16 bytes per slot. Compact only when the holes exceed
    // 1/64 of the slots or would grow the free slots by a quarter (or when
    // asked).
    const long long holes = n_slots - st->n_live;
    if (!a.force && !(holes > 0 && (holes * 64 > n_slots ||
                                    holes * 4 > a.capacity - n_slots)))
        return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket, 1u);
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= ntiles) break;
        if (a.withhold_first && tile == 0) {      // self-test: publish nothing for tile 0
            __syncthreads();
            continue;
        }
        const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
        Pos xs[kPPT];
        Mom us[kPPT];
#pragma unroll
        for (int v = 0; v < kPPT; v += kVec) {
            vload(a.xi + i0 + v, xs + v);
            vload(a.u + i0 + v, us + v);
        }
        long long ids[kPPT];
        if (a.ids) {
#pragma unroll
            for (int k = 0; k < kPPT; ++k) ids[k] = a.ids[i0 + k];
        }
        unsigned mask = 0;
#pragma unroll
        for (int k = 0; k < kPPT; ++k)
            if (i0 + k < n_slots && xs[k] >= Pos(0)) mask |= 1u << k;
        const int cnt = __popc(mask);
        // block exclusive scan of cnt
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        int wbase = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const int t = s_warp[w];
            wbase += (w < warp) ? t : 0;
            total += t;
        }
        const int excl = wbase + incl - cnt;
        if (threadIdx.x == 0) {
            unsigned long long* ts = a.tile_state;
            long long prefix = 0;
            if (tile == 0) {
                store_release(ts, pack_state(epoch, kFlagIncl, unsigned(total)));
            } else {
                store_release(ts + tile, pack_state(epoch, kFlagAgg, unsigned(total)));
                long long t = tile - 1;
                long long spins = 0;
                while (t >= 0) {
                    const unsigned long long w = load_acquire(ts + t);
                    const unsigned we = unsigned(w >> 34), wf = unsigned(w >> 32) & 3u;
                    if (we != (epoch & 0x3fffffffu) || wf == 0u) {
                        if (++spins > a.spin_limit) {
                            atomicOr(&st->flags, SCLF_FLAG_TIMEOUT);
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    prefix += static_cast<long long>(w & 0xffffffffull);
                    if (wf == kFlagIncl) break;
                    --t;
                }
                store_release(ts + tile, pack_state(epoch, kFlagIncl, unsigned(prefix + total)));
            }
            s_prefix = prefix;
            if (tile == ntiles - 1) {
                st->n_slots = prefix + total;
                st->compact_epoch = epoch + 1;
            }
        }
        __syncthreads();
        const long long dst = s_prefix + excl;
        if (!(dst == i0 && mask == ((1u << kPPT) - 1u))) {
            int r = 0;
#pragma unroll
            for (int k = 0; k < kPPT; ++k) {
                if (mask & (1u << k)) {
                    a.xi[dst + r] = xs[k];
                    a.u[dst + r] = us[k];
                    if (a.ids) a.ids[dst + r] = ids[k];
                    ++r;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

template <class Pos, class Mom>
int compact_grid_size(int device_sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_kernel<Pos, Mom>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

template <class Pos, class Mom>
cudaError_t launch_compact(const CompactArgs<Pos, Mom>& a, int grid, cudaStream_t s) {
    compact_kernel<Pos, Mom><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template int compact_grid_size<float, float>(int);
template int compact_grid_size<double, double>(int);
template int compact_grid_size<int, float>(int);
template cudaError_t launch_compact<float, float>(const CompactArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_compact<double, double>(const CompactArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_compact<int, float>(const CompactArgs<int, float>&, int, cudaStream_t);

}  // namespace sclf
