// (a6) of one PIC step: leap-frog of Eq. 3 over the cells (FP64), the gather
// table of the next step, and the per-step commit of the device counters with
// the next injection count (Gauss's law over the base half cell).
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// (a6): the field kernel, one thread per cell
// ---------------------------------------------------------------------------
// The inputs of cell j: its accumulated current, E_z, B_phi at j and its
// neighbours, E_r at nodes j and j + 1. Loading them apart from the update
// lets a thread have several cells' loads in flight.
template <class AccT>
struct CellIn {
    AccT q;
    double ez, bj, bm, bp, er0, er1;
};

template <class Real, int kAcc>
__device__ __forceinline__ void field_load(const FieldArgs<Real>& a, int j,
                                           CellIn<typename AccType<kAcc>::T>& in) {
    using AccT = typename AccType<kAcc>::T;
    const int nz = a.c.nz;
    in.q = static_cast<const AccT*>(a.jacc)[j];
    in.bj = a.b_in[j];
    in.bm = j >= 1 ? a.b_in[j - 1] : 0.0;
    in.bp = j + 1 < nz ? a.b_in[j + 1] : 0.0;
    in.ez = a.ez[j];
    in.er0 = a.er_in[j];
    in.er1 = a.er_in[j + 1];
}

// Cell j of one tube (0 <= j < Nz) from its loaded inputs; cell 0 also
// commits the tube's step.
template <class Real, int kAcc>
__device__ __forceinline__ void field_store(const FieldArgs<Real>& a, int j,
                                            const CellIn<typename AccType<kAcc>::T>& in) {
    using AccT = typename AccType<kAcc>::T;
    const int nz = a.c.nz;
    static_cast<AccT*>(a.jacc)[j] = AccT(0);
    double ssum;
    if constexpr (kAcc == kAccFixed) ssum = double(in.q) * kFixedInv;
    else ssum = in.q;
    const double J = a.c.s_over_dt * ssum;                 // J^{n+1/2}_{j+1/2}
    a.jlast[j] = J;

    const double bj = in.bj;
    const double ez1 = in.ez + a.c.dt * bj - a.c.fourpi_dt * J;
    a.ez[j] = ez1;
    // E_r at node j (node 0 stays: phi = 0 on the conducting base) ...
    const double erj = (j == 0) ? in.er0 : in.er0 - a.c.cdt * (bj - in.bm);
    // ... and at node j + 1, with the ghost B_{Nz+1/2} = B_{Nz-1/2} on top
    const double bjp = (j + 1 < nz) ? in.bp : bj;
    const double erj1 = in.er1 - a.c.cdt * (bjp - bj);
    a.er_out[j] = erj;
    if (j == a.hi - 1) a.er_out[a.hi] = erj1;     // the last node (a sub-domain's: shared)
    a.b_out[j] = bj - a.c.cdt * (erj1 - erj) - a.c.dt * ez1;

    // gather table of the next step: entry m = (E_{m-1/2}, E_{m+1/2}), ends clamped
    const Real e = static_cast<Real>(ez1);
    a.ez2[2 * j + 1] = e;
    a.ez2[2 * (j + 1)] = e;
    if (j == 0) a.ez2[0] = e;
    if (j == nz - 1) a.ez2[2 * nz + 1] = e;

    if (j == a.lo) {
        // commit of the step's counters and the next injection count (only the
        // sub-domain at the base injects)
        DevState* st = a.st;
        const long long inj = st->inj_done;
        const long long rem = static_cast<long long>(st->acc_removed);
        st->n_slots += inj;
        st->n_live += inj - rem;
        st->total_injected += inj;
        st->last_injected = inj;
        st->last_removed = rem;
        if (a.evlog) a.evlog[kLogStride * st->step + kLogRemoved] = rem;
        st->w0 = static_cast<long long>(st->acc_w0);
        long long n = 0;
        double es = 0.0;
        if (j == 0) injection_count(ez1, st->w0, a.c, &n, &es);
        st->n_inj = n;
        st->surface_field = es;
        st->acc_w0 = 0;
        st->acc_removed = 0;
        st->inj_done = 0;
        st->ticket = 0;
        st->step += 1;
    }
}

template <class Real, int kAcc>
__device__ __forceinline__ void field_cell(const FieldArgs<Real>& a, int j) {
    CellIn<typename AccType<kAcc>::T> in;
    field_load<Real, kAcc>(a, j, in);
    field_store<Real, kAcc>(a, j, in);
}

// 128 threads per block: measured 4-5 % faster than 256 on the 16384-cell
// adjoint tube (22.99 -> 21.93 ms per 2000-step forward pass), where the
// kernel is latency-bound and more blocks spread its loads over more SMs.
constexpr int kFieldBlock = 128;
template <class Real, int kAcc>
__global__ void __launch_bounds__(kFieldBlock) field_kernel(const FieldArgs<Real> a) {
    grid_dependency_wait();
    const int j = a.lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.hi) return;
    field_cell<Real, kAcc>(a, j);
}

// All tubes of a batch: kBatchCells cells per thread of the batch's cell
// space, strided by the block size so that each round is coalesced. The
// batch's grids are larger than what stays in L2 next to the particles, so a
// thread issues all its cells' loads before it updates them.
constexpr int kBatchCells = 2;

__device__ __forceinline__ FieldArgs<float> batch_field_args(const BatchTube& d, int parity) {
    FieldArgs<float> a;
    a.st = d.st;
    a.ez = d.ez;
    a.er_in = d.er[parity];
    a.er_out = d.er[parity ^ 1];
    a.b_in = d.b[parity];
    a.b_out = d.b[parity ^ 1];
    a.jacc = d.jacc;
    a.jlast = d.jlast;
    a.ez2 = d.ez2;
    a.evlog = nullptr;
    a.c = d.fc;
    a.lo = 0;
    a.hi = d.nz;
    return a;
}

__global__ void __launch_bounds__(256)
batch_field_kernel(const BatchTube* __restrict__ tubes, const int* __restrict__ cell_tube,
                   int n_cells, int parity) {
    grid_dependency_wait();
    const long long base = static_cast<long long>(blockIdx.x) * blockDim.x * kBatchCells +
                           threadIdx.x;
    int ti[kBatchCells];
#pragma unroll
    for (int k = 0; k < kBatchCells; ++k) {
        const long long g = base + static_cast<long long>(k) * blockDim.x;
        ti[k] = g < n_cells ? cell_tube[g] : -1;
    }
    // cells are numbered tube by tube, so equal first and last tubes mean
    // all of this thread's cells belong to one tube
    if (ti[kBatchCells - 1] >= 0 && ti[0] == ti[kBatchCells - 1]) {
        const BatchTube& d = tubes[ti[0]];
        const FieldArgs<float> a = batch_field_args(d, parity);
        CellIn<long long> in[kBatchCells];
#pragma unroll
        for (int k = 0; k < kBatchCells; ++k)
            field_load<float, kAccFixed>(a, static_cast<int>(base + k * blockDim.x) - d.cell0, in[k]);
#pragma unroll
        for (int k = 0; k < kBatchCells; ++k)
            field_store<float, kAccFixed>(a, static_cast<int>(base + k * blockDim.x) - d.cell0, in[k]);
    } else {
        for (int k = 0; k < kBatchCells; ++k) {
            if (ti[k] < 0) continue;
            const BatchTube& d = tubes[ti[k]];
            field_cell<float, kAccFixed>(batch_field_args(d, parity),
                                         static_cast<int>(base + k * blockDim.x) - d.cell0);
        }
    }
}

}  // namespace

template <class Real>
cudaError_t launch_field(const FieldArgs<Real>& a, int accumulate, cudaStream_t s, bool overlap) {
    const int grid = (a.hi - a.lo + kFieldBlock - 1) / kFieldBlock;
    return accumulate == kAccFixed
               ? launch_kernel(field_kernel<Real, kAccFixed>, grid, kFieldBlock, 0, s, overlap, a)
               : launch_kernel(field_kernel<Real, kAccF64>, grid, kFieldBlock, 0, s, overlap, a);
}

cudaError_t launch_batch_field(const BatchTube* tubes, const int* cell_tube, int n_cells,
                               int parity, cudaStream_t s, bool overlap) {
    const int per_block = 256 * kBatchCells;
    return launch_kernel(batch_field_kernel, (n_cells + per_block - 1) / per_block, 256, 0, s,
                         overlap, tubes, cell_tube, n_cells, parity);
}

template cudaError_t launch_field<float>(const FieldArgs<float>&, int, cudaStream_t, bool);
template cudaError_t launch_field<double>(const FieldArgs<double>&, int, cudaStream_t, bool);
}  // namespace sclf
