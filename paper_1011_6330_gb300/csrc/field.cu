// (a6) of one PIC step: leap-frog of Eq. 3 over the cells (FP64), the gather
// table of the next step, and the per-step commit of the device counters with
// the next injection count (Gauss's law over the base half cell).
#include "device_common.cuh"

namespace sclf {
namespace {

// ---------------------------------------------------------------------------
// (a6): the field kernel, one thread per cell
// ---------------------------------------------------------------------------
// Cell j of one tube (0 <= j < Nz); cell 0 also commits the tube's step.
template <class Real, int kAcc>
__device__ __forceinline__ void field_cell(const FieldArgs<Real>& a, int j) {
    using AccT = typename AccType<kAcc>::T;
    const int nz = a.c.nz;
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
        if (a.evlog) a.evlog[kLogStride * st->step + kLogRemoved] = rem;
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

template <class Real, int kAcc>
__global__ void __launch_bounds__(256) field_kernel(const FieldArgs<Real> a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.c.nz) return;
    field_cell<Real, kAcc>(a, j);
}

// All tubes of a batch: one thread per cell of the batch's cell space.
__global__ void __launch_bounds__(256)
batch_field_kernel(const BatchTube* __restrict__ tubes, const int* __restrict__ cell_tube,
                   int n_cells, int parity) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_cells) return;
    const BatchTube& d = tubes[cell_tube[g]];
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
    field_cell<float, kAccFixed>(a, g - d.cell0);
}

}  // namespace

template <class Real>
cudaError_t launch_field(const FieldArgs<Real>& a, int accumulate, cudaStream_t s) {
    const int grid = (a.c.nz + 255) / 256;
    if (accumulate == kAccFixed) field_kernel<Real, kAccFixed><<<grid, 256, 0, s>>>(a);
    else field_kernel<Real, kAccF64><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_field(const BatchTube* tubes, const int* cell_tube, int n_cells,
                               int parity, cudaStream_t s) {
    batch_field_kernel<<<(n_cells + 255) / 256, 256, 0, s>>>(tubes, cell_tube, n_cells, parity);
    return cudaGetLastError();
}

template cudaError_t launch_field<float>(const FieldArgs<float>&, int, cudaStream_t);
template cudaError_t launch_field<double>(const FieldArgs<double>&, int, cudaStream_t);
}  // namespace sclf
