// Reverse sweep of the PIC step of Sec. 2 (Figure A): the discrete adjoint
// of a recorded run with its injection counts frozen. Per step, the
// transposed leap-frog of Eq. 3 on the grid (FP64), then per particle the
// adjoints of the charge-conserving deposit, the Eq. 1 push and the
// cloud-in-cell gather, with the gather's share of the E_z adjoint reduced
// per cell by warp-aggregated runs. Also the two objectives of a run and
// their adjoint seeds.
//
// The piecewise-linear gather and deposit are differentiated inside their
// pieces: dF_j/dx = 1 for j <= x < j + 1 with F_j(x) = clamp(x - j, 0, 1),
// and dE_p/dx = E_{m+1/2} - E_{m-1/2}.
#include "device_common.cuh"

namespace sclf {
namespace {

template <class Real> struct PairT { using T = float2; };
template <> struct PairT<double> { using T = double2; };

// ---------------------------------------------------------------------------
// Eq. 3 transposed. The forward step (R = 1) is
//   E_z'  = E_z + dt B - 4 pi dt J
//   E_r'_k = E_r,k - cdt (B_k - B_{k-1})  (k = 1..Nz, ghost B_Nz = B_{Nz-1}),
//   E_r'_0 = E_r,0
//   B'    = B - cdt (E_r'_{j+1} - E_r'_j) - dt E_z'
// and, read backwards, cell j needs lambda_B of cells j-1, j, j+1 and
// lambda_Er of nodes j, j+1.
// ---------------------------------------------------------------------------
template <class Real>
__global__ void __launch_bounds__(256) adj_field_kernel(const AdjFieldArgs<Real> a) {
    grid_dependency_wait();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int nz = a.nz;
    if (j >= nz) return;
    const double cdt = a.cdt, dt = a.dt;
    const double lb_m = j >= 1 ? a.lb_in[j - 1] : 0.0;
    const double lb_j = a.lb_in[j];
    const double lb_p = j + 1 < nz ? a.lb_in[j + 1] : 0.0;
    // lambda of E_r' once B' has passed its share back: node k gets
    // + cdt lambda_B,k (k < Nz) - cdt lambda_B,{k-1} (k >= 1)
    const double le_j = a.ler_in[j] + cdt * (lb_j - lb_m);
    const double le_p = a.ler_in[j + 1] + cdt * (lb_p - lb_j);
    const double lez1 = a.lez[j] - dt * lb_j;
    a.ler_out[j] = le_j;
    if (j == nz - 1) a.ler_out[nz] = le_p;
    // B_j enters E_r'_j with -cdt (when j >= 1) and E_r'_{j+1} with +cdt
    // (when j + 1 <= Nz - 1); at the top node the ghost's two terms cancel
    double lb = lb_j + dt * lez1;
    if (j >= 1) lb -= cdt * le_j;
    if (j + 1 <= nz - 1) lb += cdt * le_p;
    a.lb_out[j] = lb;
    a.lez[j] = lez1;
    const double lj = -a.fourpi_dt * lez1;
    a.lsum[j] += lj * a.jstep[j];
    a.ls_tab[j] = static_cast<Real>(a.s_over_dt * lj);
}

// ---------------------------------------------------------------------------
// Particles: one tile of kThreads * kPPT slots per CTA pass, thread t owns
// slots [i0, i0 + kPPT) as in the forward particle kernel.
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ void adj_push_tile(const AdjPushArgs<Real>& a, long long tile,
                                              long long n_slots, long long n_tot) {
    using L = Layout<Real>;
    constexpr int kPPT = L::kPPT, kVec = L::kVec, kTile = L::kTile;
    using Pair = typename PairT<Real>::T;
    const Real nzf = a.nzf, dt = a.dt, cfl = a.cfl;
    const int nz = a.nz;
    const Pair* __restrict__ tab = reinterpret_cast<const Pair*>(a.ez2);
    const Real* __restrict__ ls = a.ls_tab;

    const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
    Real xs[kPPT], us[kPPT], lxs[kPPT], lus[kPPT];
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        vload(a.xi + i0 + v, xs + v);
        vload(a.u + i0 + v, us + v);
        vload(a.lx + i0 + v, lxs + v);
        vload(a.lu + i0 + v, lus + v);
    }
    const long long r_slots = n_slots - i0, r_tot = n_tot - i0;
    const int k_real = r_slots <= 0 ? 0 : (r_slots >= kPPT ? kPPT : int(r_slots));
    const int k_tot = r_tot <= 0 ? 0 : (r_tot >= kPPT ? kPPT : int(r_tot));
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {           // the step's new electrons start at (0, 0)
        if (k >= k_real && k < k_tot) {
            xs[k] = Real(0);
            us[k] = Real(0);
        }
    }
    // the gather's share goes to cells m-1 and m; particles sharing the
    // thread's first m (away from the clamped ends) join two per-thread runs
    const Real rkey = r_floor(xs[0] + Real(0.5));
    Real ra = Real(0), rb = Real(0);
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        const Real x = xs[k];
        const bool lv = (k < k_tot) & (x >= Real(0)) & (x < nzf);
        const Real xx = lv ? x : Real(0);
        // the forward step, recomputed with the forward kernel's operations
        const Real h = xx + Real(0.5);
        const Real mf = r_floor(h);
        const Real f = h - mf;
        const int mi = static_cast<int>(mf);
        const Pair e = checked_index(mi, nz + 1, a.flags) ? tab[mi] : Pair{};
        const Real ep = (Real(1) - f) * e.x + f * e.y;
        const Real u1 = us[k] - ep * dt;
        const Real g = r_sqrt(Real(1) + u1 * u1);
        const Real x1 = xx + r_div(u1, g) * cfl;
        const bool fin = lv & r_finite(x1);
        const bool stay = fin & (x1 >= Real(0)) & (x1 < nzf);    // still in the tube
        // (a4) J_j = (s/dt) sum [F_j(x1) - F_j(x0)]; both table reads are
        // unconditional (the index is clamped to a valid cell when unused)
        const int c1 = stay ? static_cast<int>(r_floor(x1)) : 0;
        const int c0 = static_cast<int>(r_floor(xx));
        const Real ls1 = checked_index(c1, nz, a.flags) ? ls[c1] : Real(0);
        const Real ls0 = checked_index(c0, nz, a.flags) ? ls[c0] : Real(0);
        const Real lx1 = stay ? lxs[k] + ls1 : Real(0);
        const Real lu1 = stay ? lus[k] : Real(0);
        Real lx0 = fin ? lx1 - ls0 : Real(0);
        // (a3) x1 = x0 + (u1 / gamma) cfl, d(u1 / gamma)/du1 = gamma^-3
        const Real ig = r_div(Real(1), g);
        const Real lu0 = fin ? lu1 + lx1 * cfl * (ig * ig * ig) : Real(0);
        // (a2) u1 = u0 - E_p dt, E_p = (1 - f) E_a + f E_b
        const Real lep = -dt * lu0;
        lx0 += lep * (e.y - e.x);
        const Real wa = (Real(1) - f) * lep, wb = f * lep;
        const bool common = lv & (mf == rkey) & (mf >= Real(1)) & (mf <= nzf - Real(1));
        ra += common ? wa : Real(0);
        rb += common ? wb : Real(0);
        if (lv & !common & (lep != Real(0))) {
            const int m = static_cast<int>(mf);
            const int ia = m - 1 < 0 ? 0 : m - 1;
            const int ib = m > nz - 1 ? nz - 1 : m;
            atomicAdd(a.lez + ia, static_cast<double>(wa));
            atomicAdd(a.lez + ib, static_cast<double>(wb));
        }
        lxs[k] = lx0;
        lus[k] = lu0;
    }
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        if (i0 + v < n_tot) {
            vstore(a.lx + i0 + v, lxs + v);
            vstore(a.lu + i0 + v, lus + v);
        }
    }
    const int kb = (rkey >= Real(1) && rkey <= nzf - Real(1)) ? static_cast<int>(rkey) : -1;
    warp_flush<double>(kb >= 0 ? kb - 1 : -1, static_cast<double>(ra), a.lez);
    warp_flush<double>(kb, static_cast<double>(rb), a.lez);
}

template <class Real>
__global__ void __launch_bounds__(kThreads) adj_push_kernel(const AdjPushArgs<Real> a) {
    constexpr int kTile = Layout<Real>::kTile;
    grid_dependency_wait();
    const long long n_slots = a.log[kLogSlots];
    const long long n_tot = n_slots + a.log[kLogInjected];
    const long long ntiles = (n_tot + kTile - 1) / kTile;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        adj_push_tile<Real>(a, tile, n_slots, n_tot);
}

// The same for SCLF_FIX32 positions: the forward step is recomputed exactly
// (displacement d rounded half-even to the 2^-fb grid), the rounding is
// differentiated as the identity, adjoints are in cell units.
__device__ __forceinline__ void adj_push_fix32_tile(const AdjPushFixArgs& a, long long tile,
                                                    long long n_slots, long long n_tot) {
    constexpr int kPPT = Layout<int>::kPPT, kVec = Layout<int>::kVec, kTile = Layout<int>::kTile;
    const int nz = a.nz, fb = a.fb;
    const long long top = static_cast<long long>(nz) << fb;
    const unsigned half = 1u << (fb - 1), mask = (1u << fb) - 1u;
    const float dt = a.dt, cfl = a.cfl, scale = a.scale, two_fb = a.two_fb;
    const float2* __restrict__ tab = reinterpret_cast<const float2*>(a.ez2);
    const float* __restrict__ ls = a.ls_tab;

    const long long i0 = tile * kTile + static_cast<long long>(threadIdx.x) * kPPT;
    int xs[kPPT];
    float us[kPPT], lxs[kPPT], lus[kPPT];
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        vload(a.X + i0 + v, xs + v);
        vload(a.u + i0 + v, us + v);
        vload(a.lx + i0 + v, lxs + v);
        vload(a.lu + i0 + v, lus + v);
    }
    const long long r_slots = n_slots - i0, r_tot = n_tot - i0;
    const int k_real = r_slots <= 0 ? 0 : (r_slots >= kPPT ? kPPT : int(r_slots));
    const int k_tot = r_tot <= 0 ? 0 : (r_tot >= kPPT ? kPPT : int(r_tot));
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        if (k >= k_real && k < k_tot) {
            xs[k] = 0;
            us[k] = 0.0f;
        }
    }
    const unsigned rkey = (k_tot > 0 && xs[0] >= 0)
                              ? (static_cast<unsigned>(xs[0]) + half) >> fb : 0xffffffffu;
    float ra = 0.0f, rb = 0.0f;
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        const bool lv = (k < k_tot) & (xs[k] >= 0);
        const unsigned U = lv ? static_cast<unsigned>(xs[k]) : 0u;
        const unsigned h = U + half;
        const unsigned m = h >> fb;
        const float f = __uint2float_rn(h & mask) * scale;
        const float2 e = checked_index(m, nz + 1, a.flags) ? tab[m] : float2{};
        const float ep = (1.0f - f) * e.x + f * e.y;
        const float u1 = us[k] - ep * dt;
        const float g = __fsqrt_rn(1.0f + u1 * u1);
        const float d = __fdiv_rn(u1, g) * cfl;
        const bool fin = lv & isfinite(d);
        const int inc = fin ? __float2int_rn(d * two_fb) : 0;
        const long long X1 = static_cast<long long>(U) + inc;
        const bool stay = fin & (X1 >= 0) & (X1 < top);
        const int c1 = stay ? static_cast<int>(X1 >> fb) : 0;
        const int c0 = static_cast<int>(U >> fb);
        const float ls1 = checked_index(c1, nz, a.flags) ? ls[c1] : 0.0f;
        const float ls0 = checked_index(c0, nz, a.flags) ? ls[c0] : 0.0f;
        const float lx1 = stay ? lxs[k] + ls1 : 0.0f;
        const float lu1 = stay ? lus[k] : 0.0f;
        float lx0 = fin ? lx1 - ls0 : 0.0f;
        const float ig = __fdiv_rn(1.0f, g);
        const float lu0 = fin ? lu1 + lx1 * cfl * (ig * ig * ig) : 0.0f;
        const float lep = -dt * lu0;
        lx0 += lep * (e.y - e.x);
        const float wa = (1.0f - f) * lep, wb = f * lep;
        const bool common = lv & (m == rkey) & (m >= 1u) & (m <= static_cast<unsigned>(nz - 1));
        ra += common ? wa : 0.0f;
        rb += common ? wb : 0.0f;
        if (lv & !common & (lep != 0.0f)) {
            const int ia = m < 1u ? 0 : static_cast<int>(m) - 1;
            const int ib = m > static_cast<unsigned>(nz - 1) ? nz - 1 : static_cast<int>(m);
            atomicAdd(a.lez + ia, static_cast<double>(wa));
            atomicAdd(a.lez + ib, static_cast<double>(wb));
        }
        lxs[k] = lx0;
        lus[k] = lu0;
    }
#pragma unroll
    for (int v = 0; v < kPPT; v += kVec) {
        if (i0 + v < n_tot) {
            vstore(a.lx + i0 + v, lxs + v);
            vstore(a.lu + i0 + v, lus + v);
        }
    }
    const int kb = (rkey != 0xffffffffu && rkey >= 1u && rkey <= static_cast<unsigned>(nz - 1))
                       ? static_cast<int>(rkey) : -1;
    warp_flush<double>(kb >= 0 ? kb - 1 : -1, static_cast<double>(ra), a.lez);
    warp_flush<double>(kb, static_cast<double>(rb), a.lez);
}

__global__ void __launch_bounds__(kThreads) adj_push_fix32_kernel(const AdjPushFixArgs a) {
    constexpr int kTile = Layout<int>::kTile;
    grid_dependency_wait();
    const long long n_slots = a.log[kLogSlots];
    const long long n_tot = n_slots + a.log[kLogInjected];
    const long long ntiles = (n_tot + kTile - 1) / kTile;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        adj_push_fix32_tile(a, tile, n_slots, n_tot);
}

// ---------------------------------------------------------------------------
// Objectives and seeds
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;
}

// Per block: sum of gamma over the live slots and of E_z^2 over the cells
// (fixed grid-stride assignment, so the result does not depend on timing).
template <class Pos, class Mom>
__global__ void __launch_bounds__(256) objective_partials(const Pos* xi, const Mom* u,
                                                          const DevState* st, const double* ez,
                                                          int nz, double* part) {
    __shared__ double sh[8];
    const long long n = st->n_slots;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    double sg = 0.0, se = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += stride) {
        if (xi[i] >= Pos(0)) {
            const double v = static_cast<double>(u[i]);
            sg += sqrt(1.0 + v * v);
        }
    }
    for (long long j = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; j < nz;
         j += stride)
        se += ez[j] * ez[j];
    sg = block_sum(sg, sh);
    se = block_sum(se, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sg;
        part[2 * blockIdx.x + 1] = se;
    }
}

__global__ void objective_finish(const double* part, int nblocks, const DevState* st,
                                 double dz, double* out) {
    if (threadIdx.x != 0) return;
    double sg = 0.0, se = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        sg += part[2 * b];
        se += part[2 * b + 1];
    }
    const long long live = st->n_live;
    out[0] = live > 0 ? sg / static_cast<double>(live) : 0.0;
    out[1] = sqrt(se * dz);
}

template <class Pos, class Mom>
__global__ void seed_gamma_kernel(const Pos* xi, const Mom* u, const DevState* st, Mom* lx,
                                  Mom* lu) {
    const long long n = st->n_slots;
    const long long live = st->n_live;
    const double inv = live > 0 ? 1.0 / static_cast<double>(live) : 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const bool live_slot = xi[i] >= Pos(0);
        const double v = static_cast<double>(u[i]);
        lx[i] = Mom(0);
        lu[i] = live_slot ? static_cast<Mom>(v / sqrt(1.0 + v * v) * inv) : Mom(0);
    }
}

__global__ void seed_ez_kernel(const double* ez, int nz, double dz, const double* values,
                               double* lez) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nz) return;
    const double norm = values[1];
    lez[j] = norm > 0.0 ? ez[j] * dz / norm : 0.0;
}

}  // namespace

template <class Real>
cudaError_t launch_adj_field(const AdjFieldArgs<Real>& a, cudaStream_t s, bool overlap) {
    constexpr int kBlock = 128;                // as the forward field kernel
    return launch_kernel(adj_field_kernel<Real>, (a.nz + kBlock - 1) / kBlock, kBlock, 0, s,
                         overlap, a);
}

template <class Real>
int adj_push_grid_size(int device_sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_push_kernel<Real>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

template <class Real>
cudaError_t launch_adj_push(const AdjPushArgs<Real>& a, int grid, cudaStream_t s, bool overlap) {
    return launch_kernel(adj_push_kernel<Real>, grid, kThreads, 0, s, overlap, a);
}

template <class Pos, class Mom>
cudaError_t launch_objectives(const Pos* xi, const Mom* u, const DevState* st,
                              const double* ez, int nz, double dz, double* part,
                              double* out, cudaStream_t s) {
    objective_partials<Pos, Mom><<<kObjBlocks, 256, 0, s>>>(xi, u, st, ez, nz, part);
    objective_finish<<<1, 32, 0, s>>>(part, kObjBlocks, st, dz, out);
    return cudaGetLastError();
}

template <class Pos, class Mom>
cudaError_t launch_seed_gamma(const Pos* xi, const Mom* u, const DevState* st, Mom* lx,
                              Mom* lu, cudaStream_t s) {
    seed_gamma_kernel<Pos, Mom><<<1024, 256, 0, s>>>(xi, u, st, lx, lu);
    return cudaGetLastError();
}

int adj_push_fix32_grid_size(int device_sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_push_fix32_kernel, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * device_sms;
}

cudaError_t launch_adj_push_fix32(const AdjPushFixArgs& a, int grid, cudaStream_t s,
                                  bool overlap) {
    return launch_kernel(adj_push_fix32_kernel, grid, kThreads, 0, s, overlap, a);
}

cudaError_t launch_seed_ez(const double* ez, int nz, double dz, const double* values,
                           double* lez, cudaStream_t s) {
    seed_ez_kernel<<<(nz + 255) / 256, 256, 0, s>>>(ez, nz, dz, values, lez);
    return cudaGetLastError();
}

template cudaError_t launch_adj_field<float>(const AdjFieldArgs<float>&, cudaStream_t, bool);
template cudaError_t launch_adj_field<double>(const AdjFieldArgs<double>&, cudaStream_t, bool);
template cudaError_t launch_adj_push<float>(const AdjPushArgs<float>&, int, cudaStream_t, bool);
template cudaError_t launch_adj_push<double>(const AdjPushArgs<double>&, int, cudaStream_t, bool);
template int adj_push_grid_size<float>(int);
template int adj_push_grid_size<double>(int);
template cudaError_t launch_objectives<float, float>(const float*, const float*, const DevState*,
                                                     const double*, int, double, double*, double*,
                                                     cudaStream_t);
template cudaError_t launch_objectives<double, double>(const double*, const double*,
                                                       const DevState*, const double*, int, double,
                                                       double*, double*, cudaStream_t);
template cudaError_t launch_objectives<int, float>(const int*, const float*, const DevState*,
                                                   const double*, int, double, double*, double*,
                                                   cudaStream_t);
template cudaError_t launch_seed_gamma<float, float>(const float*, const float*, const DevState*,
                                                     float*, float*, cudaStream_t);
template cudaError_t launch_seed_gamma<double, double>(const double*, const double*,
                                                       const DevState*, double*, double*,
                                                       cudaStream_t);
template cudaError_t launch_seed_gamma<int, float>(const int*, const float*, const DevState*,
                                                   float*, float*, cudaStream_t);

}  // namespace sclf
