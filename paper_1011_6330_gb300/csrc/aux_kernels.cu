// Small kernels around the step: appending particles, the base-cell weight,
// the injection count after an append, the cloud-in-cell charge density for
// diagnostics and the initial gather table.
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// Small kernels: append, base weight, ρ diagnostics, gather table
// ---------------------------------------------------------------------------
template <class Pos, class Mom>
__global__ void append_kernel(DevState* st, Pos* xi, Mom* u, long long* ids,
                              long long first, long long n, bool zero) {
    const long long id0 = st->total_injected;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (zero) { xi[first + k] = Pos(0); u[first + k] = Mom(0); }
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

// W_0 of fixed-point positions: sum over the base cell of (2^fb - X) 2^(32-fb).
__global__ void base_weight_fix32_kernel(DevState* st, const int* X, long long n, int fb) {
    long long w = 0;
    const int one = 1 << fb;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = X[i];
        if (x >= 0 && x < one) w += static_cast<long long>(one - x) << (32 - fb);
    }
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&st->acc_w0, static_cast<unsigned long long>(w));
}

template <class Pos, class Mom>
__global__ void validate_kernel(DevState* st, const Pos* xi, const Mom* u, const long long* ids,
                                long long n, double top) {
    bool bad = false;
    long long mx = -1;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double x = static_cast<double>(xi[i]);        // exact for every Pos
        if (!(x >= 0.0 && x < top) || !isfinite(static_cast<double>(u[i]))) bad = true;
        if (ids) {
            const long long id = ids[i];
            if (id < 0) bad = true;
            mx = id > mx ? id : mx;
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->load_bad, 1u);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long o = __shfl_xor_sync(kFull, mx, off);
        mx = o > mx ? o : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx >= 0) atomicMax(&st->max_id, mx);
}

__global__ void finish_append_kernel(DevState* st, const double* ez, long long n_added,
                                     FieldConsts c) {
    st->n_slots += n_added;
    st->n_live += n_added;
    st->total_injected += n_added;
    st->w0 += static_cast<long long>(st->acc_w0);
    st->acc_w0 = 0;
    long long n;
    double es;
    injection_count(ez[0], st->w0, c, &n, &es);
    st->n_inj = n;
    st->surface_field = es;
}

template <class Pos>
__global__ void rho_kernel(const Pos* xi, long long n, double* acc, int nz, double scale) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (!(xi[i] >= Pos(0))) continue;                      // hole
        const double x = double(xi[i]) * scale;
        if (!(x >= 0.0 && x < double(nz))) continue;
        const double jf = floor(x);
        const int j = static_cast<int>(jf);
        const double w = x - jf;
        atomicAdd(acc + j, 1.0 - w);
        atomicAdd(acc + j + 1, w);
    }
}

// velocity_f32 against the general-range IEEE sequence on the float32 bit
// patterns [first, first + count): out[0] counts the patterns whose results
// differ (two NaNs count as equal), out[1] keeps the smallest such pattern.
__global__ void velocity_check_kernel(unsigned first, unsigned long long count,
                                      unsigned long long* out) {
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    unsigned long long bad = 0, lowest = ~0ULL;
    for (unsigned long long i = blockIdx.x * static_cast<unsigned long long>(blockDim.x) +
                                threadIdx.x;
         i < count; i += stride) {
        const unsigned bits = first + static_cast<unsigned>(i);
        const float u = __uint_as_float(bits);
        const float a = velocity_f32(u), b = velocity_f32_ieee(u);
        const bool same = __float_as_uint(a) == __float_as_uint(b) || (isnan(a) && isnan(b));
        if (!same) {
            ++bad;
            lowest = bits < lowest ? bits : lowest;
        }
    }
    bad = warp_sum(bad);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, lowest, off);
        lowest = o < lowest ? o : lowest;
    }
    if ((threadIdx.x & 31) == 0 && bad) {
        atomicAdd(out, bad);
        atomicMin(out + 1, lowest);
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

// Per block over the live slots: count, sum of gamma, max gamma (fixed grid
// and a fixed-order finish, so the result does not depend on timing).
template <class Pos, class Mom>
__global__ void __launch_bounds__(256) particle_diag_kernel(const Pos* xi, const Mom* u,
                                                            long long n, double* part) {
    __shared__ double s_sum[8], s_max[8], s_cnt[8];
    double cnt = 0.0, sum = 0.0, mx = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (xi[i] >= Pos(0)) {
            const double v = static_cast<double>(u[i]);
            const double g = sqrt(1.0 + v * v);
            cnt += 1.0;
            sum += g;
            mx = g > mx ? g : mx;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, off);
        sum += __shfl_xor_sync(kFull, sum, off);
        const double o = __shfl_xor_sync(kFull, mx, off);
        mx = o > mx ? o : mx;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_cnt[w] = cnt; s_sum[w] = sum; s_max[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0, su = 0.0, m = 0.0;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
            c += s_cnt[k];
            su += s_sum[k];
            m = s_max[k] > m ? s_max[k] : m;
        }
        part[3 * blockIdx.x] = c;
        part[3 * blockIdx.x + 1] = su;
        part[3 * blockIdx.x + 2] = m;
    }
}

__global__ void particle_diag_finish(const double* part, int nblocks, double* out) {
    if (threadIdx.x != 0) return;
    double c = 0.0, su = 0.0, m = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        c += part[3 * b];
        su += part[3 * b + 1];
        m = part[3 * b + 2] > m ? part[3 * b + 2] : m;
    }
    out[0] = c;
    out[1] = su;
    out[2] = m;
}

int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return static_cast<int>(g < cap ? g : cap);
}

}  // namespace

template <class Pos, class Mom>
cudaError_t launch_append(DevState* st, Pos* xi, Mom* u, long long* ids, long long first,
                          long long n, bool zero_particles, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (!zero_particles && !ids) return cudaSuccess;
    append_kernel<Pos, Mom><<<grid_for(n, 256, 4096), 256, 0, s>>>(st, xi, u, ids, first, n,
                                                                   zero_particles);
    return cudaGetLastError();
}

cudaError_t launch_base_weight_fix32(DevState* st, const int* X, long long n_slots, int fb,
                                     cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    base_weight_fix32_kernel<<<grid_for(n_slots, 256, 4096), 256, 0, s>>>(st, X, n_slots, fb);
    return cudaGetLastError();
}

template <class Real>
cudaError_t launch_base_weight(DevState* st, const Real* xi, long long n_slots, cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    base_weight_kernel<Real><<<grid_for(n_slots, 256, 4096), 256, 0, s>>>(st, xi, n_slots);
    return cudaGetLastError();
}

template <class Pos, class Mom>
cudaError_t launch_particle_diag(const Pos* xi, const Mom* u, long long n, double* part,
                                 double* out, cudaStream_t s) {
    particle_diag_kernel<Pos, Mom><<<kDiagBlocks, 256, 0, s>>>(xi, u, n, part);
    particle_diag_finish<<<1, 32, 0, s>>>(part, kDiagBlocks, out);
    return cudaGetLastError();
}

template <class Pos, class Mom>
cudaError_t launch_validate(DevState* st, const Pos* xi, const Mom* u, const long long* ids,
                            long long n, double top, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    validate_kernel<Pos, Mom><<<grid_for(n, 256, 4096), 256, 0, s>>>(st, xi, u, ids, n, top);
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

cudaError_t launch_velocity_check(unsigned first, unsigned long long count,
                                  unsigned long long* out, int grid, cudaStream_t s) {
    velocity_check_kernel<<<grid, 256, 0, s>>>(first, count, out);
    return cudaGetLastError();
}

template <class Pos>
cudaError_t launch_rho(const Pos* xi, long long n_slots, double* rho_acc, int nz, double scale,
                       cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    rho_kernel<Pos><<<grid_for(n_slots, 256, 4096), 256, 0, s>>>(xi, n_slots, rho_acc, nz, scale);
    return cudaGetLastError();
}

template cudaError_t launch_append<float, float>(DevState*, float*, float*, long long*,
                                                long long, long long, bool, cudaStream_t);
template cudaError_t launch_append<double, double>(DevState*, double*, double*, long long*,
                                                  long long, long long, bool, cudaStream_t);
template cudaError_t launch_append<int, float>(DevState*, int*, float*, long long*, long long,
                                              long long, bool, cudaStream_t);
template cudaError_t launch_particle_diag<float, float>(const float*, const float*, long long,
                                                       double*, double*, cudaStream_t);
template cudaError_t launch_particle_diag<double, double>(const double*, const double*, long long,
                                                         double*, double*, cudaStream_t);
template cudaError_t launch_particle_diag<int, float>(const int*, const float*, long long,
                                                     double*, double*, cudaStream_t);
template cudaError_t launch_validate<float, float>(DevState*, const float*, const float*,
                                                  const long long*, long long, double, cudaStream_t);
template cudaError_t launch_validate<double, double>(DevState*, const double*, const double*,
                                                    const long long*, long long, double,
                                                    cudaStream_t);
template cudaError_t launch_validate<int, float>(DevState*, const int*, const float*,
                                                const long long*, long long, double, cudaStream_t);
template cudaError_t launch_base_weight<float>(DevState*, const float*, long long, cudaStream_t);
template cudaError_t launch_base_weight<double>(DevState*, const double*, long long, cudaStream_t);
template cudaError_t launch_ez_table<float>(const double*, float*, int, cudaStream_t);
template cudaError_t launch_ez_table<double>(const double*, double*, int, cudaStream_t);
template cudaError_t launch_rho<float>(const float*, long long, double*, int, double, cudaStream_t);
template cudaError_t launch_rho<double>(const double*, long long, double*, int, double, cudaStream_t);
template cudaError_t launch_rho<int>(const int*, long long, double*, int, double, cudaStream_t);
}  // namespace sclf
