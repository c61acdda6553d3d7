// (a1)-(a5) of one PIC step (Sec. 2, Figure A of arXiv:1011.6330) for tubes
// whose particle positions are 32-bit fixed point (SCLF_FIX32). The slots are
// streamed in place or (for a recorded run) into a separate output array.
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// (a1)-(a5) with SCLF_FIX32 positions: X = xi 2^fb in int32 (holes < 0),
// float32 momenta and push, the displacement rounded half-even to the 2^-fb
// grid, current fractions and the base weight as exact integers (2^-32 units).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long shl_signed(long long v, int sh) {
    return static_cast<long long>(static_cast<unsigned long long>(v) << sh);
}

// What one tile needs.
struct FixCtx {
    int* Xo;
    float* uo;
    long long* ids;
    const float2* tab;
    long long* jacc;
    unsigned int* flags;
    long long n_slots, n_tot, id0;
    int nz, fb, sh;
    unsigned half, mask;
    long long one, top;
    float dt, cfl, scale, two_fb;
    long long lo_x, hi_x;      // owned positions [lo 2^fb, hi 2^fb) (0, top: whole tube)
    const Outbox* out;         // [down, up] (device; null for a whole tube)
};

// A particle that leaves the sub-domain for a neighbour's cells (see push.cu).
__device__ __forceinline__ void emigrate_fix(const Outbox* out, int side, int X, float u,
                                             long long id, unsigned int* flags) {
    if (!out) {                                      // a whole tube has no neighbour
        atomicOr(flags, SCLF_FLAG_CAPACITY);
        return;
    }
    const Outbox& ob = out[side];
    const unsigned long long k = ob.n ? atomicAdd(ob.n, 1ULL) : ~0ULL;
    if (k < static_cast<unsigned long long>(ob.cap)) {
        static_cast<int*>(ob.x)[k] = X;
        static_cast<float*>(ob.u)[k] = u;
        if (ob.ids) ob.ids[k] = id;
    } else {
        atomicOr(flags, SCLF_FLAG_CAPACITY);
    }
}

// One tile of kThreads * kPPT slots whose thread's slots are in xs, us.
__device__ __forceinline__ void fix32_tile(const FixCtx& c, long long tile,
                                           int (&xs)[Layout<int>::kPPT],
                                           float (&us)[Layout<int>::kPPT], long long& w0_acc,
                                           long long& removed, bool& nonfinite) {
    constexpr int kPPT = Layout<int>::kPPT, kVec = Layout<int>::kVec, kTile = Layout<int>::kTile;
    const int nz = c.nz, fb = c.fb, sh = c.sh;
    const unsigned half = c.half, mask = c.mask;
    const long long one = c.one, top = c.top;
    const float dt = c.dt, cfl = c.cfl, scale = c.scale, two_fb = c.two_fb;
    const float2* __restrict__ tab = c.tab;
    long long* __restrict__ jacc = c.jacc;
    const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
    const long long r_slots = c.n_slots - i0, r_tot = c.n_tot - i0;
    const int k_real = r_slots <= 0 ? 0 : (r_slots >= kPPT ? kPPT : int(r_slots));
    const int k_tot = r_tot <= 0 ? 0 : (r_tot >= kPPT ? kPPT : int(r_tot));
    if (k_real < k_tot) {                        // (a1) new electrons at the base
#pragma unroll
        for (int k = 0; k < kPPT; ++k) {
            if (k >= k_real && k < k_tot) {
                xs[k] = 0;
                us[k] = 0.0f;
                if (c.ids) c.ids[i0 + k] = c.id0 + (i0 + k - c.n_slots);
            }
        }
    }
    if (k_tot < kPPT) {                          // padding past the last slot: a hole
#pragma unroll
        for (int k = 0; k < kPPT; ++k)
            if (k >= k_tot) xs[k] = -1;
    }
    // Runs on two cells, c_r and c_r + 1: c_r is the lower of the cells of
    // the thread's first and last slots (sorted slots at ~100 particles per
    // cell often span two cells), when it lies in [1, hi - 2] (hi = Nz for a
    // whole tube, else the sub-domain's end; so Nz >= 3 and fb <= 29). With
    // A = c_r 2^fb, a particle is common when U - A and U1 - A are both below
    // 2^(fb+1): it starts and ends in c_r or c_r + 1 (live, cell >= 1, inside
    // the tube and the sub-domain). In 2^-fb units its current on c_r is
    // F_cr(X1) - F_cr(X) = min(U1 - A, 2^fb) - min(U - A, 2^fb) and the rest
    // of its increment falls on c_r + 1, so the runs keep the sum of the
    // increments and the sum of the parts on c_r. Without a run the bound is
    // 0 and no particle is common. (Measured: 0.308 against 0.323 ms for the
    // run on the first slot's cell alone on the 1e8-particle tube, 0.677
    // against 0.896 ms on the death-line batch.)
    // A hole carries X = -1 (removals and padding write exactly that; loaded
    // slots have no holes), so U = 2^32 - 1: its gather index wraps to 0 and
    // U - A >= 2^32 - 2^31 > 2^(fb+1), so it is never common and needs no
    // test of its own on the common path.
    int xr = xs[0];
    const int xl = xs[kPPT - 1];
    xr = (xr < 0 || (xl >= 0 && xl < xr)) ? xl : xr;
    const bool has_run = xr >= static_cast<int>(one) && xr < c.hi_x - one;
    const unsigned A = static_cast<unsigned>(xr) & ~mask;
    const unsigned one_u = 1u << fb, bound = has_run ? 2u << fb : 0u;
    // The runs are summed modulo 2^32: every particle's increment and part on
    // c_r are added, and those of particles that are not common are taken
    // back out on their own path (exact, and cheaper than a select each).
    unsigned s_inc = 0, s_low = 0;
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        const unsigned U = static_cast<unsigned>(xs[k]);
        // (a2) h = X + 2^(fb-1): m = h >> fb, f = (h mod 2^fb) 2^-fb
        const unsigned h = U + half;
        const float f = __uint2float_rn(h & mask) * scale;
        const unsigned m = h >> fb;
        const float2 e = checked_index(m, nz + 1, c.flags) ? tab[m] : float2{};
        const float ep = (1.0f - f) * e.x + f * e.y;
        // (a3) Eq. 1, then the displacement on the 2^-fb grid
        const float u1 = us[k] - ep * dt;
        const float d = velocity_f32(u1) * cfl;
        // |v| <= 1 and c dt < dz: a finite d has |d| <= 1 (NaN fails the test)
        const bool fin = fabsf(d) <= 1.0f;
        const int inc = __float2int_rn(d * two_fb);  // |inc| <= 2^fb
        // X1 = X + inc in 32-bit arithmetic: X < Nz 2^fb <= 2^31 and
        // |inc| <= 2^fb keep U + inc away from wrapping for cells >= 1
        const unsigned U1 = U + static_cast<unsigned>(inc);
        // (a4) the common particle's current joins the runs
        // both offsets below 2^(fb+1), a power of two: so is their OR
        const unsigned t0 = U - A, t1 = U1 - A;
        const bool common = fin & ((t0 | t1) < bound);
        const int low = static_cast<int>(min(t1, one_u)) - static_cast<int>(min(t0, one_u));
        s_inc += static_cast<unsigned>(inc);
        s_low += static_cast<unsigned>(low);
        if (common) {
            xs[k] = static_cast<int>(U1);
            us[k] = u1;
            continue;
        }
        s_inc -= static_cast<unsigned>(inc);     // not in the runs: taken back out
        s_low -= static_cast<unsigned>(low);
        const int XX = xs[k];
        if (XX < 0) {                            // a hole stays one
            if constexpr (kChecked) {
                if (XX != -1) atomicOr(c.flags, SCLF_FLAG_BOUNDS);
            }
            continue;
        }
        const long long X1 = static_cast<long long>(XX) + inc;
        const long long c1 = X1 >> fb;
        const unsigned c0 = U >> fb;
        if (!fin) {
            nonfinite = true;
            ++removed;
            xs[k] = -1;
            us[k] = 0.0f;
            continue;
        }
        const long long b0 = static_cast<long long>(c0) << fb;
        const long long f0a = min(max(static_cast<long long>(XX) - b0, 0LL), one);
        const long long f1a = min(max(X1 - b0, 0LL), one);
        const long long qa = shl_signed(f1a - f0a, sh);
        if (qa && checked_index(c0, nz, c.flags)) acc_add(jacc + c0, qa);
        if (c1 != static_cast<long long>(c0) && c1 >= 0 && c1 < nz) {
            const long long b1 = c1 << fb;
            const long long f0b = min(max(static_cast<long long>(XX) - b1, 0LL), one);
            const long long f1b = min(max(X1 - b1, 0LL), one);
            const long long qb = shl_signed(f1b - f0b, sh);
            if (qb) acc_add(jacc + static_cast<int>(c1), qb);
        }
        // (a5) removal at the ends; base-cell weight for the next injection
        if (X1 >= c.lo_x && X1 < c.hi_x) {
            xs[k] = static_cast<int>(X1);
            us[k] = u1;
            if (c1 == 0) w0_acc += shl_signed(one - X1, sh);
        } else if (X1 >= 0 && X1 < top) {         // to a neighbouring sub-domain
            emigrate_fix(c.out, X1 < c.lo_x ? 0 : 1, static_cast<int>(X1), u1,
                         c.ids ? c.ids[i0 + k] : -1LL, c.flags);
            xs[k] = -1;
            us[k] = 0.0f;
        } else {
            ++removed;
            xs[k] = -1;
            us[k] = 0.0f;
        }
    }
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        if (i0 + v < c.n_tot) {
            vstore(c.Xo + i0 + v, xs + v);
            vstore(c.uo + i0 + v, us + v);
        }
    }
    const int key = has_run ? static_cast<int>(A >> fb) : -1;
    const int key2 = has_run ? key + 1 : -1;
    int ra = static_cast<int>(s_low), rb = static_cast<int>(s_inc - s_low);
    if constexpr (kChecked) {
        if (ra != 0 && !checked_index(key, nz, c.flags)) ra = 0;
        if (rb != 0 && !checked_index(key2, nz, c.flags)) rb = 0;
    }
    // |ra|, |rb| <= 8 2^fb per lane: 32-lane segment sums fit 32 bits up to fb = 22
    if (fb <= 22) {
        warp_flush2_i32(key, ra, rb, jacc, sh);
    } else {
        warp_flush<long long>(key, shl_signed(ra, sh), jacc);
        warp_flush<long long>(key2, shl_signed(rb, sh), jacc);
    }
}

// The particle kernel of SCLF_FIX32 tubes. kStages == 1: each tile's slots
// are loaded straight into registers; kStages >= 2: the next tiles stream
// through a ring of shared-memory stages by bulk asynchronous copies (TMA).
// At least 4 CTAs of 256 threads per SM: 0.343 ms per step of the 1e8-particle
// frame-dragging tube and 3.80 ms of the 2^30-particle large tube, against
// 0.362 and 4.05 ms at 3 CTAs per SM and 1.613 ms (2^28 particles) with no
// bound.
constexpr int kFix32MinBlocks = 4;
template <int kStages>
__global__ void __launch_bounds__(kThreads, kFix32MinBlocks) push_fix32_kernel(const PushFixArgs a) {
    constexpr int kPPT = Layout<int>::kPPT, kVec = Layout<int>::kVec, kTile = Layout<int>::kTile;
    grid_dependency_wait();
    // The CTA's first tile is loaded before the step's counters are read: the
    // slot arrays are padded to whole tiles, so a tile that starts below the
    // capacity lies inside them, and the counters only decide which of its
    // slots are live. In small tubes, where a CTA has one tile, the two
    // loads' latencies overlap.
    int xs[kPPT], xn[kPPT];
    float us[kPPT], un[kPPT];
    if constexpr (kStages == 1) {
        if (static_cast<long long>(blockIdx.x) * kTile < a.capacity) {
            const long long i0 = static_cast<long long>(blockIdx.x) * kTile +
                                 static_cast<long long>(threadIdx.x) * kPPT;
#pragma unroll
            for (int v = 0; v < kPPT; v += kVec) {
                vload(a.X + i0 + v, xs + v);
                vload(a.u + i0 + v, us + v);
            }
        }
    }
    DevState* st = a.st;
    const long long n_slots = st->n_slots;
    const long long n_req = a.replay ? a.replay[kLogStride * st->step + kLogInjected] : st->n_inj;
    long long room = a.capacity - n_slots;
    room = room > 0 ? room : 0;
    const long long n_inj = n_req < room ? n_req : room;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->inj_done = n_inj;
        st->slots_processed += static_cast<unsigned long long>(n_slots + n_inj);
        if (n_inj < n_req) atomicOr(&st->flags, SCLF_FLAG_CAPACITY);
        if (a.evlog) {
            a.evlog[kLogStride * st->step + kLogSlots] = n_slots;
            a.evlog[kLogStride * st->step + kLogInjected] = n_inj;
        }
    }
    FixCtx c;
    c.Xo = a.Xo;
    c.uo = a.uo;
    c.ids = a.ids;
    c.tab = reinterpret_cast<const float2*>(a.ez2);
    c.jacc = a.jacc;
    c.flags = &st->flags;
    c.n_slots = n_slots;
    c.n_tot = n_slots + n_inj;
    c.id0 = st->total_injected;
    c.nz = a.nz;
    c.fb = a.fb;
    c.sh = 32 - a.fb;
    c.half = 1u << (a.fb - 1);
    c.mask = (1u << a.fb) - 1u;
    c.one = 1LL << a.fb;
    c.top = static_cast<long long>(a.nz) << a.fb;    // first position past the tube
    c.dt = a.dt;
    c.cfl = a.cfl;
    c.scale = a.scale;
    c.two_fb = a.two_fb;
    c.lo_x = static_cast<long long>(a.lo) << a.fb;
    c.hi_x = static_cast<long long>(a.hi) << a.fb;
    c.out = a.out;
    const long long ntiles = (c.n_tot + kTile - 1) / kTile;

    long long w0_acc = 0;
    long long removed = 0;
    bool nonfinite = false;
    if constexpr (kStages == 1) {
        // the next tile's slots are loaded into registers before this tile's
        // work, so every warp keeps loads in flight while it computes
        // (measured on one box: 0.3146 against 0.3171 ms on the 1e8 tube,
        // 3.487 against 3.572 ms on the 2^30 tube, although ptxas spills
        // 36 bytes at 4 CTAs per SM; at 3 CTAs per SM, without spills, it
        // is 0.370 ms)
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const long long nt = tile + gridDim.x;
            if (nt < ntiles) {
                const long long i1 = nt * kTile + static_cast<long long>(threadIdx.x) * kPPT;
#pragma unroll
                for (int v = 0; v < kPPT; v += kVec) {
                    vload(a.X + i1 + v, xn + v);
                    vload(a.u + i1 + v, un + v);
                }
            }
            fix32_tile(c, tile, xs, us, w0_acc, removed, nonfinite);
#pragma unroll
            for (int k = 0; k < kPPT; ++k) { xs[k] = xn[k]; us[k] = un[k]; }
        }
    } else {
        extern __shared__ __align__(128) unsigned char ring_smem[];
        const TileRing<int, float, kTile, kStages> ring{ring_smem};
        ring_tiles<kPPT, kVec>(ring, a.X, a.u, ntiles, &st->flags,
                               [&](long long tile, int(&xs)[kPPT], float(&us)[kPPT]) {
                                   fix32_tile(c, tile, xs, us, w0_acc, removed, nonfinite);
                               });
    }

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

// A batch of SCLF_FIX32 tubes in one launch: persistent CTAs walk the batch's
// tile space (tiles of kThreads * 8 slots); every tile belongs to one tube and
// is pushed with that tube's constants, read from its descriptor (the next
// tile's tube index one tile ahead, as in the FP32 batch kernel).
__global__ void __launch_bounds__(kThreads, kFix32MinBlocks)
batch_push_fix32_kernel(const BatchTube* __restrict__ tubes, const int* __restrict__ tile_tube,
                        long long n_tiles) {
    constexpr int kPPT = Layout<int>::kPPT, kVec = Layout<int>::kVec, kTile = Layout<int>::kTile;
    grid_dependency_wait();
    long long w0 = 0, removed = 0;
    bool nonfinite = false;
    int ti = blockIdx.x < n_tiles ? tile_tube[blockIdx.x] : 0;
    for (long long g = blockIdx.x; g < n_tiles; g += gridDim.x) {
        const BatchTube& d = tubes[ti];
        const long long gn = g + gridDim.x;
        ti = gn < n_tiles ? tile_tube[gn] : 0;
        const long long local = g - d.tile0;
        const long long n_slots = d.n_slots, n_tot = d.n_tot;
        if (local == 0 && threadIdx.x == 0) record_injection(d.st, n_tot - n_slots, d.n_req, nullptr);
        if (local * kTile >= n_tot) continue;          // the same for the whole CTA
        FixCtx c;
        const int fb = d.fb;
        c.Xo = reinterpret_cast<int*>(d.xi);
        c.uo = d.u;
        c.ids = d.ids;
        c.tab = reinterpret_cast<const float2*>(d.ez2);
        c.jacc = d.jacc;
        c.flags = &d.st->flags;
        c.n_slots = n_slots;
        c.n_tot = n_tot;
        c.id0 = d.id0;
        c.nz = d.nz;
        c.fb = fb;
        c.sh = 32 - fb;
        c.half = 1u << (fb - 1);
        c.mask = (1u << fb) - 1u;
        c.one = 1LL << fb;
        c.top = static_cast<long long>(d.nz) << fb;
        c.dt = d.dt;
        c.cfl = d.cfl;
        c.scale = __int_as_float((127 - fb) << 23);   // 2^-fb
        c.two_fb = __int_as_float((127 + fb) << 23);  // 2^fb
        c.lo_x = 0;
        c.hi_x = c.top;
        c.out = nullptr;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(tubes + ti));
        const long long i0 = local * kTile + static_cast<long long>(threadIdx.x) * kPPT;
        int xs[kPPT];
        float us[kPPT];
#pragma unroll
        for (int v = 0; v < kPPT; v += kVec) {
            vload(c.Xo + i0 + v, xs + v);
            vload(d.u + i0 + v, us + v);
        }
        fix32_tile(c, local, xs, us, w0, removed, nonfinite);
        flush_tube_counters(d.st, w0, removed, nonfinite);
    }
}

size_t fix32_smem_bytes(int stages) {
    constexpr int kTile = Layout<int>::kTile;
    switch (stages) {
        case 2: return TileRing<int, float, kTile, 2>::kBytes;
        case 3: return TileRing<int, float, kTile, 3>::kBytes;
        case 4: return TileRing<int, float, kTile, 4>::kBytes;
        default: return 0;
    }
}

template <int kStages>
int fix32_grid_of(int device_sms) {
    const size_t smem = fix32_smem_bytes(kStages);
    cudaFuncSetAttribute(push_fix32_kernel<kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_fix32_kernel<kStages>, kThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

}  // namespace

int push_fix32_grid_size(int stages, int device_sms) {
    switch (stages) {
        case 1: return fix32_grid_of<1>(device_sms);
        case 3: return fix32_grid_of<3>(device_sms);
        case 4: return fix32_grid_of<4>(device_sms);
        default: return fix32_grid_of<2>(device_sms);
    }
}

int batch_push_fix32_grid_size(int device_sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_push_fix32_kernel, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

cudaError_t launch_batch_push_fix32(const BatchTube* tubes, const int* tile_tube,
                                    long long n_tiles, int grid, cudaStream_t s, bool overlap) {
    return launch_kernel(batch_push_fix32_kernel, grid, kThreads, 0, s, overlap, tubes, tile_tube,
                         n_tiles);
}

cudaError_t launch_push_fix32(const PushFixArgs& a, int stages, int grid, cudaStream_t s,
                              bool overlap) {
    const size_t smem = fix32_smem_bytes(stages);
    switch (stages) {
        case 1: return launch_kernel(push_fix32_kernel<1>, grid, kThreads, 0, s, overlap, a);
        case 3: return launch_kernel(push_fix32_kernel<3>, grid, kThreads, smem, s, overlap, a);
        case 4: return launch_kernel(push_fix32_kernel<4>, grid, kThreads, smem, s, overlap, a);
        default: return launch_kernel(push_fix32_kernel<2>, grid, kThreads, smem, s, overlap, a);
    }
}

}  // namespace sclf
