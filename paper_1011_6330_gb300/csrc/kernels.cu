// sm_103a kernels of one PIC step (Sec. 2, Figure A of arXiv:1011.6330).
//
//  push_kernel     (a1)-(a5): injection of the pending electrons as virtual
//                  slots, cloud-in-cell gather of E_z, the Eq. 1 push, the
//                  charge-conserving current deposit, removal at the tube
//                  ends and the base-cell weight for the next injection.
//                  Persistent CTAs stream the particle slots in place.
//  field_kernel    (a6): leap-frog of Eq. 3 over the cells, plus the
//                  per-step commit of the device counters and the next
//                  injection count (Gauss's law over the base half cell).
//  compact_kernel  stable in-place removal of holes (single pass, decoupled
//                  look-back), run every few steps.
//
// Compiled with --fmad=false: every floating-point operation is rounded on
// its own, in the order written, so the particle arithmetic is the same
// IEEE sequence in float32 or float64 that the step's definition states.
#include <cstdint>
#include <type_traits>

#include "sclf_internal.h"

namespace sclf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kAccFixed = SCLF_ACC_FIXED64;
constexpr int kAccF64 = SCLF_ACC_FP64;

template <class Real> struct Vec;
template <> struct Vec<float> { using T = float4; };
template <> struct Vec<double> { using T = double2; };

__device__ __forceinline__ void vload(const float* p, float* r) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void vload(const double* p, double* r) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void vstore(float* p, const float* r) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(r[0], r[1], r[2], r[3]));
}
__device__ __forceinline__ void vstore(double* p, const double* r) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r[0], r[1]));
}

// Round x * 2^32 to the nearest integer, ties to even (|x| <= 1 here).
__device__ __forceinline__ long long to_fixed(float x) {
    return __float2ll_rn(x * 4294967296.0f);
}
__device__ __forceinline__ long long to_fixed(double x) {
    return __double2ll_rn(x * 4294967296.0);
}

template <class Real> __device__ __forceinline__ Real clamp01(Real v) {
    return fmin(fmax(v, Real(0)), Real(1));
}
__device__ __forceinline__ float clamp01(float v) {
    return fminf(fmaxf(v, 0.0f), 1.0f);
}

// F_j(x1) - F_j(x0), F_j(x) = clamp(x - j, 0, 1): the fraction of a
// particle's charge that crossed node j during the step.
template <class Real>
__device__ __forceinline__ Real frac_delta(Real x0, Real x1, int j) {
    const Real jf = Real(j);
    return clamp01(x1 - jf) - clamp01(x0 - jf);
}

template <int kAcc> struct AccType { using T = long long; };
template <> struct AccType<kAccF64> { using T = double; };

template <int kAcc, class Real>
__device__ __forceinline__ typename AccType<kAcc>::T to_acc(Real d) {
    if constexpr (kAcc == kAccFixed) return to_fixed(d);
    else return double(d);
}

__device__ __forceinline__ void acc_add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p),
              static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void acc_add(double* p, double v) { atomicAdd(p, v); }

// Warp-wide flush of per-lane (cell, value) runs: an inclusive segmented
// scan over lanes with equal consecutive keys, then one atomic per segment.
// Keys < 0 mean "no run".
template <class AccT>
__device__ __forceinline__ void warp_flush(int key, AccT val, AccT* acc) {
    const int lane = threadIdx.x & 31;
    const int kprev = __shfl_up_sync(kFull, key, 1);
    const bool head = lane == 0 || kprev != key;
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned le = heads & (kFull >> (31 - lane));
    const int start = 31 - __clz(le);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const AccT o = __shfl_up_sync(kFull, val, off);
        if (lane - off >= start) val += o;
    }
    const int knext = __shfl_down_sync(kFull, key, 1);
    const bool tail = lane == 31 || knext != key;
    if (tail && key >= 0 && val != AccT(0)) acc_add(acc + key, val);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Number of electrons to inject (Sec. 2): E_s at the surface from Gauss's
// law over the base half cell, E_s = E_{1/2} - 4 pi s W_0 + 2 pi dz rho_GJ,0;
// N = max(0, round-half-even(-E_s / (4 pi |s|))).
__device__ __forceinline__ void injection_count(double ez_half, long long w0,
                                                const FieldConsts& c,
                                                long long* n, double* es) {
    const double wsum = double(w0) * kFixedInv;
    const double e = (ez_half - c.four_pi_s * wsum) + c.two_pi_dz_rho0;
    const double r = rint(-e / c.sheet);
    *es = e;
    *n = r > 0.0 ? (r < 4.0e18 ? static_cast<long long>(r) : 4000000000000000000LL) : 0;
}

// ---------------------------------------------------------------------------
// (a1)-(a5): the particle kernel
// ---------------------------------------------------------------------------
template <class Real, int kAcc>
__global__ void __launch_bounds__(kThreads)
push_kernel(const PushArgs<Real> a) {
    using L = Layout<Real>;
    constexpr int kPPT = L::kPPT, kVec = L::kVec, kTile = L::kTile;
    using AccT = typename AccType<kAcc>::T;
    AccT* __restrict__ jacc = static_cast<AccT*>(a.jacc);

    DevState* st = a.st;
    const long long n_slots = st->n_slots;
    const long long n_req = st->n_inj;
    long long room = a.capacity - n_slots;
    room = room > 0 ? room : 0;
    const long long n_inj = n_req < room ? n_req : room;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->inj_done = n_inj;
        st->slots_processed += static_cast<unsigned long long>(n_slots + n_inj);
        if (n_inj < n_req) atomicOr(&st->flags, SCLF_FLAG_CAPACITY);
    }
    const long long n_tot = n_slots + n_inj;
    const long long id0 = st->total_injected;
    const long long ntiles = (n_tot + kTile - 1) / kTile;

    long long w0_acc = 0;
    long long removed = 0;
    bool nonfinite = false;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
        Real xs[kPPT], us[kPPT];
#pragma unroll
        for (int v = 0; v < kPPT; v += kVec) {
            vload(a.xi + i0 + v, xs + v);
            vload(a.u + i0 + v, us + v);
        }
        int run_cell = -1;
        AccT run_acc = AccT(0);
#pragma unroll
        for (int k = 0; k < kPPT; ++k) {
            const long long i = i0 + k;
            Real x = xs[k], uu = us[k];
            bool live;
            if (i < n_slots) {
                live = x >= Real(0);                 // holes carry xi < 0
            } else if (i < n_tot) {                  // (a1) new electron at the base
                x = Real(0);
                uu = Real(0);
                live = true;
                if (a.ids) a.ids[i] = id0 + (i - n_slots);
            } else {
                live = false;                        // padding
            }
            if (!live) continue;

            // (a2) cloud-in-cell gather from the (E_{m-1/2}, E_{m+1/2}) table
            const Real h = x + Real(0.5);
            const Real mf = floor(h);
            const Real f = h - mf;
            int m = static_cast<int>(mf);
            m = m < 0 ? 0 : (m > a.nz ? a.nz : m);
            const Real ea = a.ez2[2 * m];
            const Real eb = a.ez2[2 * m + 1];
            const Real ep = (Real(1) - f) * ea + f * eb;
            // (a3) Eq. 1, q/m = -1, c = 1
            const Real u1 = uu - ep * a.dt;
            const Real g = sqrt(Real(1) + u1 * u1);
            const Real x1 = x + (u1 / g) * a.cfl;

            if (!(isfinite(x1) && isfinite(u1))) {
                nonfinite = true;
                ++removed;
                xs[k] = Real(-1);
                us[k] = Real(0);
                continue;
            }
            // (a4) charge-conserving deposit into cells floor(x) and floor(x1)
            const int c0 = static_cast<int>(floor(x));
            const int c1 = static_cast<int>(floor(x1));
            {
                const Real d = frac_delta(x, x1, c0);
                if (c0 != run_cell) {
                    if (run_cell >= 0 && run_acc != AccT(0)) acc_add(jacc + run_cell, run_acc);
                    run_cell = c0;
                    run_acc = AccT(0);
                }
                run_acc += to_acc<kAcc>(d);
            }
            if (c1 != c0 && c1 >= 0 && c1 < a.nz) {
                const AccT q = to_acc<kAcc>(frac_delta(x, x1, c1));
                if (q != AccT(0)) acc_add(jacc + c1, q);
            }
            // (a5) removal at the ends; base-cell weight for the next injection
            if (x1 >= Real(0) && x1 < a.nzf) {
                xs[k] = x1;
                us[k] = u1;
                if (x1 < Real(1)) w0_acc += to_fixed(Real(1) - x1);
            } else {
                ++removed;
                xs[k] = Real(-1);
                us[k] = Real(0);
            }
        }
#pragma unroll
        for (int v = 0; v < kPPT; v += kVec) {
            if (i0 + v < n_tot) {
                vstore(a.xi + i0 + v, xs + v);
                vstore(a.u + i0 + v, us + v);
            }
        }
        warp_flush<AccT>(run_cell, run_acc, jacc);
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
// (a6): the field kernel, one thread per cell
// ---------------------------------------------------------------------------
template <class Real, int kAcc>
__global__ void __launch_bounds__(256) field_kernel(const FieldArgs<Real> a) {
    using AccT = typename AccType<kAcc>::T;
    const int nz = a.c.nz;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nz) return;
    AccT* jacc = static_cast<AccT*>(a.jacc);
    const AccT q = jacc[j];
    jacc[j] = AccT(0);
    double ssum;
    if constexpr (kAcc == kAccFixed) ssum = double(q) * kFixedInv;
    else ssum = q;
    const double J = a.c.s_over_dt * ssum;                 // J^{n+1/2}_{j+1/2}
    a.jlast[j] = J;

    const double bj = a.b_in[j];
    const double ez1 = a.ez[j] + a.c.dt * bj - a.c.fourpi_dt * J;
    a.ez[j] = ez1;
    // E_r at node j (node 0 stays: phi = 0 on the conducting base) ...
    const double erj = (j == 0) ? a.er_in[0]
                                : a.er_in[j] - a.c.cdt * (bj - a.b_in[j - 1]);
    // ... and at node j + 1, with the ghost B_{Nz+1/2} = B_{Nz-1/2} on top
    const double bjp = (j + 1 < nz) ? a.b_in[j + 1] : bj;
    const double erj1 = a.er_in[j + 1] - a.c.cdt * (bjp - bj);
    a.er_out[j] = erj;
    if (j == nz - 1) a.er_out[nz] = erj1;
    a.b_out[j] = bj - a.c.cdt * (erj1 - erj) - a.c.dt * ez1;

    // gather table of the next step: entry m = (E_{m-1/2}, E_{m+1/2}), ends clamped
    const Real e = static_cast<Real>(ez1);
    a.ez2[2 * j + 1] = e;
    a.ez2[2 * (j + 1)] = e;
    if (j == 0) a.ez2[0] = e;
    if (j == nz - 1) a.ez2[2 * nz + 1] = e;

    if (j == 0) {
        // commit of the step's counters and the next injection count
        DevState* st = a.st;
        const long long inj = st->inj_done;
        const long long rem = static_cast<long long>(st->acc_removed);
        st->n_slots += inj;
        st->n_live += inj - rem;
        st->total_injected += inj;
        st->last_injected = inj;
        st->last_removed = rem;
        st->w0 = static_cast<long long>(st->acc_w0);
        long long n;
        double es;
        injection_count(ez1, st->w0, a.c, &n, &es);
        st->n_inj = n;
        st->surface_field = es;
        st->acc_w0 = 0;
        st->acc_removed = 0;
        st->inj_done = 0;
        st->ticket = 0;
        st->step += 1;
    }
}

// ---------------------------------------------------------------------------
// In-place stable compaction (decoupled look-back)
// ---------------------------------------------------------------------------
constexpr unsigned kFlagAgg = 1u, kFlagIncl = 2u;
constexpr long long kSpinLimit = 1LL << 22;

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

template <class Real>
__global__ void __launch_bounds__(kThreads) compact_kernel(const CompactArgs<Real> a) {
    using L = Layout<Real>;
    constexpr int kPPT = L::kPPT, kVec = L::kVec, kTile = L::kTile;
    __shared__ long long s_tile;
    __shared__ int s_warp[kThreads / 32];
    __shared__ long long s_prefix;

    DevState* st = a.st;
    const long long n_slots = st->n_slots;
    const unsigned epoch = st->compact_epoch;
    const long long ntiles = (n_slots + kTile - 1) / kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket, 1u);
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= ntiles) break;
        const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
        Real xs[kPPT], us[kPPT];
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
            if (i0 + k < n_slots && xs[k] >= Real(0)) mask |= 1u << k;
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
                        if (++spins > kSpinLimit) {
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

// ---------------------------------------------------------------------------
// Small kernels: append, base weight, ρ diagnostics, gather table
// ---------------------------------------------------------------------------
template <class Real>
__global__ void append_kernel(DevState* st, Real* xi, Real* u, long long* ids,
                              long long first, long long n, bool zero) {
    const long long id0 = st->total_injected;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (zero) { xi[first + k] = Real(0); u[first + k] = Real(0); }
        if (ids) ids[first + k] = id0 + k;
    }
}

template <class Real>
__global__ void base_weight_kernel(DevState* st, const Real* xi, long long n) {
    long long w = 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const Real x = xi[i];
        if (x >= Real(0) && x < Real(1)) w += to_fixed(Real(1) - x);
    }
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&st->acc_w0, static_cast<unsigned long long>(w));
}

__global__ void finish_append_kernel(DevState* st, const double* ez, long long n_added,
                                     FieldConsts c) {
    st->n_slots += n_added;
    st->n_live += n_added;
    st->total_injected += n_added;
    st->w0 = static_cast<long long>(st->acc_w0);
    st->acc_w0 = 0;
    long long n;
    double es;
    injection_count(ez[0], st->w0, c, &n, &es);
    st->n_inj = n;
    st->surface_field = es;
}

template <class Real>
__global__ void rho_kernel(const Real* xi, long long n, double* acc, int nz) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double x = double(xi[i]);
        if (!(x >= 0.0 && x < double(nz))) continue;
        const double jf = floor(x);
        const int j = static_cast<int>(jf);
        const double w = x - jf;
        atomicAdd(acc + j, 1.0 - w);
        atomicAdd(acc + j + 1, w);
    }
}

template <class Real>
__global__ void ez_table_kernel(const double* ez, Real* ez2, int nz) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > nz) return;
    const int lo = m - 1 < 0 ? 0 : m - 1;
    const int hi = m > nz - 1 ? nz - 1 : m;
    ez2[2 * m] = static_cast<Real>(ez[lo]);
    ez2[2 * m + 1] = static_cast<Real>(ez[hi]);
}

int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return static_cast<int>(g < cap ? g : cap);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class Real>
int push_grid_size(int accumulate, int device_sms) {
    int per_sm = 0;
    if (accumulate == kAccFixed)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_kernel<Real, kAccFixed>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_kernel<Real, kAccF64>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

template <class Real>
cudaError_t launch_push(const PushArgs<Real>& a, int accumulate, int grid, cudaStream_t s) {
    if (accumulate == kAccFixed) push_kernel<Real, kAccFixed><<<grid, kThreads, 0, s>>>(a);
    else push_kernel<Real, kAccF64><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_field(const FieldArgs<Real>& a, int accumulate, cudaStream_t s) {
    const int grid = (a.c.nz + 255) / 256;
    if (accumulate == kAccFixed) field_kernel<Real, kAccFixed><<<grid, 256, 0, s>>>(a);
    else field_kernel<Real, kAccF64><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <class Real>
int compact_grid_size(int device_sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_kernel<Real>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

template <class Real>
cudaError_t launch_compact(const CompactArgs<Real>& a, int grid, cudaStream_t s) {
    compact_kernel<Real><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_append(DevState* st, Real* xi, Real* u, long long* ids, long long first,
                          long long n, bool zero_particles, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (!zero_particles && !ids) return cudaSuccess;
    append_kernel<Real><<<grid_for(n, 256, 4096), 256, 0, s>>>(st, xi, u, ids, first, n,
                                                               zero_particles);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_base_weight(DevState* st, const Real* xi, long long n_slots, cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    base_weight_kernel<Real><<<grid_for(n_slots, 256, 4096), 256, 0, s>>>(st, xi, n_slots);
    return cudaGetLastError();
}

cudaError_t launch_finish_append(DevState* st, const double* ez, long long n_added,
                                 FieldConsts c, cudaStream_t s) {
    finish_append_kernel<<<1, 1, 0, s>>>(st, ez, n_added, c);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_ez_table(const double* ez, Real* ez2, int nz, cudaStream_t s) {
    ez_table_kernel<Real><<<(nz + 1 + 255) / 256, 256, 0, s>>>(ez, ez2, nz);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_rho(const Real* xi, long long n_slots, double* rho_acc, int nz,
                       cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    rho_kernel<Real><<<grid_for(n_slots, 256, 4096), 256, 0, s>>>(xi, n_slots, rho_acc, nz);
    return cudaGetLastError();
}

#define SCLF_INSTANTIATE(R)                                                                  \
    template int push_grid_size<R>(int, int);                                                \
    template cudaError_t launch_push<R>(const PushArgs<R>&, int, int, cudaStream_t);         \
    template cudaError_t launch_field<R>(const FieldArgs<R>&, int, cudaStream_t);            \
    template int compact_grid_size<R>(int);                                                  \
    template cudaError_t launch_compact<R>(const CompactArgs<R>&, int, cudaStream_t);        \
    template cudaError_t launch_append<R>(DevState*, R*, R*, long long*, long long,          \
                                          long long, bool, cudaStream_t);                    \
    template cudaError_t launch_base_weight<R>(DevState*, const R*, long long, cudaStream_t); \
    template cudaError_t launch_ez_table<R>(const double*, R*, int, cudaStream_t);           \
    template cudaError_t launch_rho<R>(const R*, long long, double*, int, cudaStream_t);

SCLF_INSTANTIATE(float)
SCLF_INSTANTIATE(double)

}  // namespace sclf
