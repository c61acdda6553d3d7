// (a1)-(a5) of one PIC step (Sec. 2, Figure A of arXiv:1011.6330): the
// particle kernel. Injection of the pending electrons as virtual slots,
// cloud-in-cell gather of E_z, the Eq. 1 push, the charge-conserving current
// deposit, removal at the tube ends and the base-cell weight for the next
// injection. Persistent CTAs stream the particle slots, in place or (for a
// recorded run) into a separate output array.
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// (a1)-(a5): the particle kernel
// ---------------------------------------------------------------------------
template <class Real> struct PairOf { using T = float2; };
template <> struct PairOf<double> { using T = double2; };

// Current fraction of a particle that stays in cell j >= 1 (the common path):
// F_j(x1) - F_j(x0). For float32 positions x0, x1 lie in one binade (cells
// never straddle a power of two for j >= 1), so x1 - x0 is exact, and it is a
// multiple of 2^-23: (x1 - x0) 2^31 is an exact float32 integer and one 32-bit
// conversion gives the same 2^-32-unit difference as quantising both F first.
template <int kAcc>
__device__ __forceinline__ typename AccType<kAcc>::T common_frac(float x0, float x1, float jf) {
    if constexpr (kAcc == kAccFixed)
        return static_cast<long long>(__float2int_rn((x1 - x0) * 2147483648.0f)) * 2;
    else return frac_acc_in_cell<kAcc>(x0, x1, jf);
}
template <int kAcc>
__device__ __forceinline__ typename AccType<kAcc>::T common_frac(double x0, double x1, double jf) {
    return frac_acc_in_cell<kAcc>(x0, x1, jf);
}

// Adds the warp's per-lane runs (cell key, sum) to the current. A float32
// run of exact x1 - x0 terms (multiples of 2^-20, below 16) is first
// converted to 2^-20 units exactly (below 2^24); the segmented sums of up to
// 32 lanes then stay below 2^29 and are scanned in 32-bit integers, and
// each segment's total goes to the 2^-32-unit accumulator shifted by 12.
// kWarpReduce: a warp whose lanes share one key takes one warp reduction
// (dense sorted tubes); without it every flush is the segmented scan (the
// batches' sparser tubes, where such warps are rare and the test costs).
template <bool kFloatRun, bool kWarpReduce, class AccT, class RunT>
__device__ __forceinline__ void flush_run(int key, RunT r, int nz, unsigned int* flags,
                                          AccT* jacc) {
    if constexpr (kFloatRun) {
        int q = __float2int_rn(r * 1048576.0f);
        if constexpr (kChecked)
            if (q != 0 && !checked_index(key, nz, flags)) q = 0;
        if constexpr (kWarpReduce) warp_flush_i32(key, q, jacc, 12);
        else warp_scan_flush_i32(key, q, jacc, 12);
    } else {
        if constexpr (kChecked)
            if (r != AccT(0) && !checked_index(key, nz, flags)) r = AccT(0);
        warp_flush<AccT>(key, r, jacc);
    }
}

// What one tile of one tube needs.
template <class Real, class AccT>
struct TileCtx {
    Real* xi;
    Real* u;
    Real* xo;                  // pushed slots are stored here (xi: in place)
    Real* uo;
    long long* ids;
    const typename PairOf<Real>::T* tab;
    AccT* jacc;
    unsigned int* flags;       // the tube's status word (bounds-checked builds)
    long long n_slots, n_tot, id0;
    Real nzf, dt, cfl;
    int nz;
    Real lof, hif;             // owned cells [lof, hif) (a sub-domain; 0, nzf: whole tube)
    const Outbox* out;         // [down, up] (device), read only when a particle leaves [lof, hif)
};

// A particle that leaves the sub-domain for a neighbour's cells: appended to
// that side's outbox (an overflow sets SCLF_FLAG_CAPACITY and loses it).
template <class P, class M>
__device__ __forceinline__ void emigrate(const Outbox* out, int side, P x, M u, long long id,
                                         unsigned int* flags) {
    if (!out) {                                      // a whole tube has no neighbour
        atomicOr(flags, SCLF_FLAG_CAPACITY);
        return;
    }
    const Outbox& ob = out[side];
    const unsigned long long k = ob.n ? atomicAdd(ob.n, 1ULL) : ~0ULL;
    if (k < static_cast<unsigned long long>(ob.cap)) {
        static_cast<P*>(ob.x)[k] = x;
        static_cast<M*>(ob.u)[k] = u;
        if (ob.ids) ob.ids[k] = id;
    } else {
        atomicOr(flags, SCLF_FLAG_CAPACITY);
    }
}

// One tile of kThreads * kPPT slots: thread t owns slots [i0, i0 + kPPT)
// (kPPT defaults to the precision's layout; the batched kernel varies it).
// Adds the tile's base weight, removals and non-finite flag to the caller's
// counters.
// The tile body: the thread's kPPT slots are already in xs, us.
template <class Real, int kAcc, int kPPT = Layout<Real>::kPPT, bool kTwoRuns = false,
          bool kWarpReduce = true>
__device__ __forceinline__ void push_tile_body(const TileCtx<Real, typename AccType<kAcc>::T>& c,
                                               long long tile, Real (&xs)[kPPT],
                                               Real (&us)[kPPT], long long& w0_acc,
                                               long long& removed, bool& nonfinite) {
    using L = Layout<Real>;
    constexpr int kVec = L::kVec, kTile = kThreads * kPPT;
    static_assert(kPPT % kVec == 0, "whole vectors per thread");
    using AccT = typename AccType<kAcc>::T;
    using Pair = typename PairOf<Real>::T;
    const Real nzf = c.nzf, dt = c.dt, cfl = c.cfl;
    const int nz = c.nz;
    const Pair* __restrict__ tab = c.tab;
    AccT* __restrict__ jacc = c.jacc;

    const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
    // slots [i0, i0 + k_real) hold particles or holes, [k_real, k_tot)
    // are this step's new electrons, the rest is padding
    const long long r_slots = c.n_slots - i0, r_tot = c.n_tot - i0;
    const int k_real = r_slots <= 0 ? 0 : (r_slots >= kPPT ? kPPT : int(r_slots));
    const int k_tot = r_tot <= 0 ? 0 : (r_tot >= kPPT ? kPPT : int(r_tot));
    if (k_real < k_tot) {                        // (a1) new electrons at the base
#pragma unroll
        for (int k = 0; k < kPPT; ++k) {
            if (k >= k_real && k < k_tot) {
                xs[k] = Real(0);
                us[k] = Real(0);
                if (c.ids) c.ids[i0 + k] = c.id0 + (i0 + k - c.n_slots);
            }
        }
    }
    if (k_tot < kPPT) {                          // padding past the last slot: a hole
#pragma unroll
        for (int k = 0; k < kPPT; ++k)
            if (k >= k_tot) xs[k] = Real(-1);
    }
    // The common particle stays inside the cell of the thread's first
    // particle, away from the base cells and the top: its current
    // fraction joins a per-thread run without any branch. Everything
    // else (crossing a node, the base cells, leaving the tube, another
    // cell, a non-finite result) takes the rare branch. With kTwoRuns the
    // cell of the thread's last particle keeps a second run (sorted
    // particles at ~100 per cell often put a thread's particles in two
    // cells). A run key is a cell >= kRunMin or the sentinel -2, which no
    // floor(xx) equals (xx >= 0): a common particle then has x0f == x1f >=
    // kRunMin, so it is live and 1 <= x1 < Nz without further tests.
    //
    // Float32 positions with the fixed-point current keep the run as a
    // float32 sum of x1 - x0: for cells j >= 8 every x1 - x0 is exact and a
    // multiple of 2^-20, |x1 - x0| < 1 (c dt < dz), so every partial sum of
    // up to 16 terms is below 16 and exact, and sum * 2^20 is an integer
    // below 2^24: one conversion at the flush gives the same 2^-32-unit
    // total as converting each term.
    constexpr bool kFloatRun = std::is_same<Real, float>::value && kAcc == kAccFixed;
    static_assert(!kFloatRun || kPPT <= 16, "float run: at most 16 terms");
    using RunT = typename std::conditional<kFloatRun, float, AccT>::type;
    constexpr Real kRunMin = kFloatRun ? Real(8) : Real(1);
    const Real rkey = xs[0] >= kRunMin ? r_floor(xs[0]) : Real(-2);
    const Real rkey2 = kTwoRuns ? (xs[kPPT - 1] >= kRunMin ? r_floor(xs[kPPT - 1]) : Real(-2))
                                : rkey;
    RunT ra = RunT(0), rb = RunT(0);
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        const Real x = xs[k];
        const bool lv = (x >= Real(0)) & (x < nzf);   // holes and padding carry xi < 0
        const Real xx = lv ? x : Real(0);
        // (a2) cloud-in-cell gather from the (E_{m-1/2}, E_{m+1/2}) table;
        // 0 <= xx < Nz keeps m in [0, Nz]
        const Real h = xx + Real(0.5);
        const Real mf = r_floor(h);
        const Real f = h - mf;
        const int m = static_cast<int>(mf);
        const Pair e = checked_index(m, nz + 1, c.flags) ? tab[m] : Pair{};
        const Real ep = (Real(1) - f) * e.x + f * e.y;
        // (a3) Eq. 1, q/m = -1, c = 1
        const Real u1 = us[k] - ep * dt;
        const Real x1 = xx + r_velocity(u1) * cfl;
        // (a4) charge-conserving deposit into cells floor(x) and floor(x1)
        const Real x0f = r_floor(xx);
        const Real x1f = r_floor(x1);
        const bool first = x0f == rkey;
        const bool common = (x1f == x0f) & (first | (kTwoRuns & (x0f == rkey2)));
        RunT q0;
        if constexpr (kFloatRun) q0 = x1 - xx;
        else q0 = common_frac<kAcc>(xx, x1, x0f);
        ra += (common & first) ? q0 : RunT(0);
        if constexpr (kTwoRuns) rb += (common & !first) ? q0 : RunT(0);
        if (lv & !common) {
            if (!r_finite(x1)) {                 // a non-finite u1 makes x1 non-finite
                nonfinite = true;
                ++removed;
                xs[k] = Real(-1);
                us[k] = Real(0);
            } else {
                const int c0 = static_cast<int>(x0f);
                AccT qa = frac_acc_in_cell<kAcc>(xx, x1, x0f);
                if (x1f != x0f) {
                    qa = frac_acc<kAcc>(xx, x1, c0);
                    const int c1 = static_cast<int>(x1f);
                    if (c1 >= 0 && c1 < nz) {
                        const AccT q1 = frac_acc<kAcc>(xx, x1, c1);
                        if (q1 != AccT(0)) acc_add(jacc + c1, q1);
                    }
                }
                if (qa != AccT(0) && checked_index(c0, nz, c.flags)) acc_add(jacc + c0, qa);
                // (a5) removal at the ends; base-cell weight for the next injection
                if (x1 >= c.lof && x1 < c.hif) {
                    xs[k] = x1;
                    us[k] = u1;
                    if (x1 < Real(1)) w0_acc += to_fixed(Real(1) - x1);
                } else if (x1 >= Real(0) && x1 < nzf) {   // to a neighbouring sub-domain
                    emigrate<Real, Real>(c.out, x1 < c.lof ? 0 : 1, x1, u1,
                                         c.ids ? c.ids[i0 + k] : -1LL, c.flags);
                    xs[k] = Real(-1);
                    us[k] = Real(0);
                } else {
                    ++removed;
                    xs[k] = Real(-1);
                    us[k] = Real(0);
                }
            }
        } else {
            xs[k] = common ? x1 : xs[k];
            us[k] = common ? u1 : us[k];
        }
    }
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        if (i0 + v < c.n_tot) {
            vstore(c.xo + i0 + v, xs + v);
            vstore(c.uo + i0 + v, us + v);
        }
    }
    const int key = rkey >= Real(0) ? static_cast<int>(rkey) : -1;
    flush_run<kFloatRun, kWarpReduce, AccT>(key, ra, nz, c.flags, jacc);
    if constexpr (kTwoRuns) {
        const int key2 = rkey2 >= Real(0) && rkey2 != rkey ? static_cast<int>(rkey2) : -1;
        flush_run<kFloatRun, kWarpReduce, AccT>(key2, rb, nz, c.flags, jacc);
    }
}

// A tile with its slots loaded straight from global memory into registers.
template <class Real, int kAcc, int kPPT = Layout<Real>::kPPT, bool kTwoRuns = false,
          bool kWarpReduce = true>
__device__ __forceinline__ void push_tile(const TileCtx<Real, typename AccType<kAcc>::T>& c,
                                          long long tile, long long& w0_acc, long long& removed,
                                          bool& nonfinite) {
    constexpr int kVec = Layout<Real>::kVec, kTile = kThreads * kPPT;
    const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
    Real xs[kPPT], us[kPPT];
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        vload(c.xi + i0 + v, xs + v);
        vload(c.u + i0 + v, us + v);
    }
    push_tile_body<Real, kAcc, kPPT, kTwoRuns, kWarpReduce>(c, tile, xs, us, w0_acc, removed,
                                                            nonfinite);
}

// Injection bookkeeping of a step: the requested count (the tube's own, or
// a replayed one) clipped to the free slots. The caller that owns the tube's
// first tile records it.
__device__ __forceinline__ long long requested_injection(const DevState* st,
                                                         const long long* replay) {
    return replay ? replay[kLogStride * st->step + kLogInjected] : st->n_inj;
}
__device__ __forceinline__ long long clipped_injection(const DevState* st, long long capacity,
                                                       long long n_req) {
    long long room = capacity - st->n_slots;
    room = room > 0 ? room : 0;
    return n_req < room ? n_req : room;
}

// The particle kernel. kStages == 1: each tile's slots are loaded straight
// into registers. kStages >= 2: the tiles a CTA will process next stream into
// a ring of kStages shared-memory stages by bulk asynchronous copies (TMA)
// while it computes, and each thread takes its slots from there.
// 4 CTAs of 256 threads per SM (at most 64 registers): measured fastest on
// the 1e8-particle tube (0.320 ms against 0.353 ms at 3 and 0.441 ms with
// no bound, where the compiler takes 103 registers; 4 particles per thread
// at 5 CTAs per SM took 0.323 ms against 0.314 ms for 8 at 4).
constexpr int kPushMinBlocks = 4;
template <class Real, int kAcc, int kStages>
__global__ void __launch_bounds__(kThreads, kPushMinBlocks)
push_kernel(const PushArgs<Real> a) {
    constexpr int kTile = Layout<Real>::kTile;
    constexpr int kPPT1 = Layout<Real>::kPPT, kVec1 = Layout<Real>::kVec;
    using AccT = typename AccType<kAcc>::T;
    grid_dependency_wait();
    // The CTA's first tile is loaded before the step's counters are read (the
    // slot arrays are padded to whole tiles, and the counters only decide
    // which of the tile's slots are live): in small tubes, where a CTA has one
    // tile, the two loads' latencies overlap.
    Real xs[kPPT1], us[kPPT1];
    if constexpr (kStages == 1) {
        if (static_cast<long long>(blockIdx.x) * kTile < a.capacity) {
            const long long i0 = static_cast<long long>(blockIdx.x) * kTile +
                                 static_cast<long long>(threadIdx.x) * kPPT1;
#pragma unroll
            for (int v = 0; v < kPPT1; v += kVec1) {
                vload(a.xi + i0 + v, xs + v);
                vload(a.u + i0 + v, us + v);
            }
        }
    }
    DevState* st = a.st;
    const long long n_req = requested_injection(st, a.replay);
    const long long n_inj = clipped_injection(st, a.capacity, n_req);
    if (blockIdx.x == 0 && threadIdx.x == 0) record_injection(st, n_inj, n_req, a.evlog);
    TileCtx<Real, AccT> c;
    c.xi = a.xi;
    c.u = a.u;
    c.xo = a.xo;
    c.uo = a.uo;
    c.ids = a.ids;
    c.tab = reinterpret_cast<const typename PairOf<Real>::T*>(a.ez2);
    c.jacc = static_cast<AccT*>(a.jacc);
    c.flags = &st->flags;
    c.n_slots = st->n_slots;
    c.n_tot = c.n_slots + n_inj;
    c.id0 = st->total_injected;
    c.nzf = a.nzf;
    c.dt = a.dt;
    c.cfl = a.cfl;
    c.nz = a.nz;
    c.lof = static_cast<Real>(a.lo);
    c.hif = static_cast<Real>(a.hi);
    c.out = a.out;
    const long long ntiles = (c.n_tot + kTile - 1) / kTile;

    long long w0_acc = 0;
    long long removed = 0;
    bool nonfinite = false;
    if constexpr (kStages == 1) {
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (tile != blockIdx.x) {
                const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT1;
#pragma unroll
                for (int v = 0; v < kPPT1; v += kVec1) {
                    vload(a.xi + i0 + v, xs + v);
                    vload(a.u + i0 + v, us + v);
                }
            }
            push_tile_body<Real, kAcc>(c, tile, xs, us, w0_acc, removed, nonfinite);
        }
    } else {
        constexpr int kPPT = Layout<Real>::kPPT, kVec = Layout<Real>::kVec;
        extern __shared__ __align__(128) unsigned char ring_smem[];
        const TileRing<Real, Real, kTile, kStages> ring{ring_smem};
        ring_tiles<kPPT, kVec>(ring, c.xi, c.u, ntiles, &st->flags,
                               [&](long long tile, Real(&xs)[kPPT], Real(&us)[kPPT]) {
                                   push_tile_body<Real, kAcc>(c, tile, xs, us, w0_acc, removed,
                                                              nonfinite);
                               });
    }

    // block totals of the removal count and W_0
    __shared__ long long s_w0[kThreads / 32], s_rm[kThreads / 32];
    __shared__ int s_nf;
    if (threadIdx.x == 0) s_nf = 0;
    __syncthreads();
    if (nonfinite) s_nf = 1;
    w0_acc = warp_sum(w0_acc);
    removed = warp_sum(removed);
    if ((threadIdx.x & 31) == 0) {
        s_w0[threadIdx.x >> 5] = w0_acc;
        s_rm[threadIdx.x >> 5] = removed;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long w = 0, r = 0;
        for (int i = 0; i < kThreads / 32; ++i) { w += s_w0[i]; r += s_rm[i]; }
        if (w) atomicAdd(&st->acc_w0, static_cast<unsigned long long>(w));
        if (r) atomicAdd(&st->acc_removed, static_cast<unsigned long long>(r));
        if (s_nf) atomicOr(&st->flags, SCLF_FLAG_NONFINITE);
    }
}



// ---------------------------------------------------------------------------
// The same step for a batch of independent tubes (FP32 particles, fixed-point
// current) in one launch: persistent CTAs walk the batch's tile space, every
// tile belongs to one tube and is pushed with that tube's constants.
// ---------------------------------------------------------------------------

template <int kPPT, int kMinBlocks, bool kTwoRuns>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
batch_push_kernel(const BatchTube* __restrict__ tubes, const int* __restrict__ tile_tube,
                  long long n_tiles) {
    constexpr int kTile = kThreads * kPPT;
    grid_dependency_wait();
    long long w0 = 0, removed = 0;
    bool nonfinite = false;
    // The tube of the next tile is loaded one tile ahead; the tube's step
    // counters come with its descriptor (batch_refresh_kernel), so a tile's
    // particle loads wait for one descriptor read only.
    int ti = blockIdx.x < n_tiles ? tile_tube[blockIdx.x] : 0;
    for (long long g = blockIdx.x; g < n_tiles; g += gridDim.x) {
        const BatchTube& d = tubes[ti];
        const long long gn = g + gridDim.x;
        ti = gn < n_tiles ? tile_tube[gn] : 0;
        const long long local = g - d.tile0;
        TileCtx<float, long long> c;
        c.n_slots = d.n_slots;
        c.n_tot = d.n_tot;
        if (local == 0 && threadIdx.x == 0)
            record_injection(d.st, c.n_tot - c.n_slots, d.n_req, nullptr);
        if (local * kTile >= c.n_tot) continue;          // the same for the whole CTA
        c.xi = d.xi;
        c.u = d.u;
        c.xo = d.xi;
        c.uo = d.u;
        c.ids = d.ids;
        c.tab = reinterpret_cast<const float2*>(d.ez2);
        c.jacc = d.jacc;
        c.flags = &d.st->flags;
        c.id0 = d.id0;
        c.nzf = d.nzf;
        c.dt = d.dt;
        c.cfl = d.cfl;
        c.nz = d.nz;
        c.lof = 0.0f;
        c.hif = d.nzf;
        c.out = nullptr;
        // the next tile's descriptor line into L1 while this tile computes
        asm volatile("prefetch.global.L1 [%0];" ::"l"(tubes + ti));
        push_tile<float, kAccFixed, kPPT, kTwoRuns, false>(c, local, w0, removed, nonfinite);
        flush_tube_counters(d.st, w0, removed, nonfinite);
    }
}

// The same with the tubes' constants in the parameter space; only the step
// counters come from the descriptors.
template <int kPPT, int kMinBlocks, bool kTwoRuns>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
batch_push_const_kernel(const __grid_constant__ BatchConstTable k,
                        const BatchTube* __restrict__ tubes, const int* __restrict__ tile_tube,
                        long long n_tiles) {
    constexpr int kTile = kThreads * kPPT;
    grid_dependency_wait();
    long long w0 = 0, removed = 0;
    bool nonfinite = false;
    int ti = blockIdx.x < n_tiles ? tile_tube[blockIdx.x] : 0;
    for (long long g = blockIdx.x; g < n_tiles; g += gridDim.x) {
        const BatchConst& kc = k.t[ti];
        const BatchTube& d = tubes[ti];
        const long long gn = g + gridDim.x;
        ti = gn < n_tiles ? tile_tube[gn] : 0;
        const long long local = g - kc.tile0;
        TileCtx<float, long long> c;
        c.n_slots = d.n_slots;
        c.n_tot = d.n_tot;
        if (local == 0 && threadIdx.x == 0)
            record_injection(kc.st, c.n_tot - c.n_slots, d.n_req, nullptr);
        if (local * kTile >= c.n_tot) continue;          // the same for the whole CTA
        c.xi = kc.xi;
        c.u = kc.u;
        c.xo = kc.xi;
        c.uo = kc.u;
        c.ids = kc.ids;
        c.tab = reinterpret_cast<const float2*>(kc.ez2);
        c.jacc = kc.jacc;
        c.flags = &kc.st->flags;
        c.id0 = d.id0;
        c.nzf = kc.nzf;
        c.dt = kc.dt;
        c.cfl = kc.cfl;
        c.nz = kc.nz;
        c.lof = 0.0f;
        c.hif = kc.nzf;
        c.out = nullptr;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(tubes + ti));
        push_tile<float, kAccFixed, kPPT, kTwoRuns, false>(c, local, w0, removed, nonfinite);
        flush_tube_counters(kc.st, w0, removed, nonfinite);
    }
}

__global__ void batch_refresh_kernel(BatchTube* tubes, int n_tubes) {
    grid_dependency_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tubes) return;
    BatchTube& d = tubes[i];
    const DevState* st = d.st;
    const long long n_slots = st->n_slots, n_req = st->n_inj, id0 = st->total_injected;
    long long room = d.capacity - n_slots;
    room = room > 0 ? room : 0;
    d.n_slots = n_slots;
    d.n_tot = n_slots + (n_req < room ? n_req : room);
    d.id0 = id0;
    d.n_req = n_req;
}

// Every tube's committed counters in the public tube_stats layout, one
// thread per tube, for a single device-to-host copy.
__global__ void batch_status_kernel(const BatchTube* tubes, int n_tubes, tube_stats* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tubes) return;
    const DevState* st = tubes[i].st;
    tube_stats s;
    s.step = st->step;
    s.n_particles = st->n_live;
    s.n_slots = st->n_slots;
    s.total_injected = st->total_injected;
    s.last_injected = st->last_injected;
    s.last_removed = st->last_removed;
    s.pending_injection = st->n_inj;
    s.surface_field = st->surface_field;
    s.flags = st->flags;
    s.reserved = 0;
    out[i] = s;
}

// The batched kernel's shapes, (particles per thread, CTAs per SM in the
// launch bounds, runs per thread); batch_autotune picks one per batch by
// timing.
template <int kPPT, int kMinBlocks, bool kTwoRuns>
int batch_grid_of(int sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_push_kernel<kPPT, kMinBlocks, kTwoRuns>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

template <int kPPT, int kMinBlocks, bool kTwoRuns>
int batch_const_grid_of(int sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_push_const_kernel<kPPT, kMinBlocks, kTwoRuns>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

// Dynamic shared memory of the particle kernel with a ring of `stages`.
template <class Real>
size_t push_smem_bytes(int stages) {
    constexpr int kTile = Layout<Real>::kTile;
    switch (stages) {
        case 2: return TileRing<Real, Real, kTile, 2>::kBytes;
        case 3: return TileRing<Real, Real, kTile, 3>::kBytes;
        case 4: return TileRing<Real, Real, kTile, 4>::kBytes;
        default: return 0;
    }
}

template <class Real, int kAcc, int kStages>
int push_grid_of(int device_sms) {
    const size_t smem = push_smem_bytes<Real>(kStages);
    cudaFuncSetAttribute(push_kernel<Real, kAcc, kStages>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_kernel<Real, kAcc, kStages>,
                                                  kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

template <class Real, int kAcc>
int push_grid_acc(int stages, int device_sms) {
    switch (stages) {
        case 1: return push_grid_of<Real, kAcc, 1>(device_sms);
        case 3: return push_grid_of<Real, kAcc, 3>(device_sms);
        case 4: return push_grid_of<Real, kAcc, 4>(device_sms);
        default: return push_grid_of<Real, kAcc, 2>(device_sms);
    }
}

template <class Real, int kAcc>
cudaError_t launch_push_acc(const PushArgs<Real>& a, int stages, int grid, cudaStream_t s,
                            bool overlap) {
    const size_t smem = push_smem_bytes<Real>(stages);
    switch (stages) {
        case 1: return launch_kernel(push_kernel<Real, kAcc, 1>, grid, kThreads, 0, s, overlap, a);
        case 3: return launch_kernel(push_kernel<Real, kAcc, 3>, grid, kThreads, smem, s, overlap, a);
        case 4: return launch_kernel(push_kernel<Real, kAcc, 4>, grid, kThreads, smem, s, overlap, a);
        default: return launch_kernel(push_kernel<Real, kAcc, 2>, grid, kThreads, smem, s, overlap, a);
    }
}

}  // namespace

template <class Real>
int push_grid_size(int accumulate, int stages, int device_sms) {
    return accumulate == kAccFixed ? push_grid_acc<Real, kAccFixed>(stages, device_sms)
                                   : push_grid_acc<Real, kAccF64>(stages, device_sms);
}

template <class Real>
cudaError_t launch_push(const PushArgs<Real>& a, int accumulate, int stages, int grid,
                        cudaStream_t s, bool overlap) {
    return accumulate == kAccFixed ? launch_push_acc<Real, kAccFixed>(a, stages, grid, s, overlap)
                                   : launch_push_acc<Real, kAccF64>(a, stages, grid, s, overlap);
}

cudaError_t launch_batch_refresh(BatchTube* tubes, int n_tubes, cudaStream_t s, bool overlap) {
    return launch_kernel(batch_refresh_kernel, (n_tubes + 127) / 128, 128, 0, s, overlap, tubes,
                         n_tubes);
}

cudaError_t launch_batch_status(const BatchTube* tubes, int n_tubes, tube_stats* out,
                                cudaStream_t s) {
    batch_status_kernel<<<(n_tubes + 127) / 128, 128, 0, s>>>(tubes, n_tubes, out);
    return cudaGetLastError();
}

int batch_push_grid_size(int variant, int device_sms) {
    switch (variant) {
        case 1: return batch_grid_of<8, 3, false>(device_sms);
        case 2: return batch_grid_of<4, 4, false>(device_sms);
        case 3: return batch_grid_of<8, 4, true>(device_sms);
        case 4: return batch_grid_of<8, 3, true>(device_sms);
        case 5: return batch_grid_of<16, 2, true>(device_sms);
        default: return batch_grid_of<8, 4, false>(device_sms);
    }
}

cudaError_t launch_batch_push(const BatchTube* tubes, const int* tile_tube, long long n_tiles,
                              int grid, int variant, cudaStream_t s, bool overlap) {
#define SCLF_BATCH_LAUNCH(P, M, T) \
    return launch_kernel(batch_push_kernel<P, M, T>, grid, kThreads, 0, s, overlap, tubes, \
                         tile_tube, n_tiles)
    switch (variant) {
        case 1: SCLF_BATCH_LAUNCH(8, 3, false);
        case 2: SCLF_BATCH_LAUNCH(4, 4, false);
        case 3: SCLF_BATCH_LAUNCH(8, 4, true);
        case 4: SCLF_BATCH_LAUNCH(8, 3, true);
        case 5: SCLF_BATCH_LAUNCH(16, 2, true);
        default: SCLF_BATCH_LAUNCH(8, 4, false);
    }
#undef SCLF_BATCH_LAUNCH
}

int batch_push_const_grid_size(int variant, int device_sms) {
    switch (variant) {
        case 1: return batch_const_grid_of<8, 3, false>(device_sms);
        case 2: return batch_const_grid_of<4, 4, false>(device_sms);
        case 3: return batch_const_grid_of<8, 4, true>(device_sms);
        case 4: return batch_const_grid_of<8, 3, true>(device_sms);
        case 5: return batch_const_grid_of<16, 2, true>(device_sms);
        default: return batch_const_grid_of<8, 4, false>(device_sms);
    }
}

cudaError_t launch_batch_push_const(const BatchConstTable& k, const BatchTube* tubes,
                                    const int* tile_tube, long long n_tiles, int grid,
                                    int variant, cudaStream_t s, bool overlap) {
#define SCLF_BATCH_LAUNCH(P, M, T) \
    return launch_kernel(batch_push_const_kernel<P, M, T>, grid, kThreads, 0, s, overlap, k, \
                         tubes, tile_tube, n_tiles)
    switch (variant) {
        case 1: SCLF_BATCH_LAUNCH(8, 3, false);
        case 2: SCLF_BATCH_LAUNCH(4, 4, false);
        case 3: SCLF_BATCH_LAUNCH(8, 4, true);
        case 4: SCLF_BATCH_LAUNCH(8, 3, true);
        case 5: SCLF_BATCH_LAUNCH(16, 2, true);
        default: SCLF_BATCH_LAUNCH(8, 4, false);
    }
#undef SCLF_BATCH_LAUNCH
}

template int push_grid_size<float>(int, int, int);
template int push_grid_size<double>(int, int, int);
template cudaError_t launch_push<float>(const PushArgs<float>&, int, int, int, cudaStream_t,
                                       bool);
template cudaError_t launch_push<double>(const PushArgs<double>&, int, int, int, cudaStream_t,
                                        bool);
}  // namespace sclf
