// Internal declarations shared by the host side and the kernels of the
// sclf_tube library. Not part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sclf_tube.h"

namespace sclf {

// Particle tiles: a CTA of kThreads threads handles kThreads * PPT
// consecutive slots, each thread PPT consecutive ones.
constexpr int kThreads = 256;
template <class Real> struct Layout;
template <> struct Layout<float> {
    static constexpr int kVec = 4;          // float4 loads
    static constexpr int kPPT = 8;          // particles per thread
    static constexpr int kTile = kThreads * kPPT;
};
template <> struct Layout<double> {
    static constexpr int kVec = 2;          // double2 loads
    static constexpr int kPPT = 4;
    static constexpr int kTile = kThreads * kPPT;
};
template <> struct Layout<int> {            // fixed-point positions (int32)
    static constexpr int kVec = 4;          // int4 loads
    static constexpr int kPPT = 8;
    static constexpr int kTile = kThreads * kPPT;
};
constexpr int kMaxTile = kThreads * 16;

// Fractional bits of SCLF_FIX32 positions: the largest fb with Nz 2^fb <= 2^31.
inline int fix32_bits(long long nz) {
    int b = 0;
    while ((1LL << b) < nz) ++b;        // b = ceil(log2 Nz)
    return 31 - b;
}

// 2^32: quantum of the fixed-point accumulators (current fractions and the
// base-cell weight W_0).
constexpr double kFixedScale = 4294967296.0;
constexpr double kFixedInv = 1.0 / 4294967296.0;

// Device-resident counters of one tube. The particle kernel reads only the
// "committed" block and writes only the "accumulated" block; the field
// kernel's first thread folds the latter into the former once per step.
struct DevState {
    // committed (valid between steps)
    long long n_slots;          // slots in use: live particles + holes
    long long n_live;           // live particles
    long long n_inj;            // electrons the next step injects
    long long total_injected;   // IDs handed out
    long long step;             // completed steps
    long long w0;               // base-cell weight W_0 (2^-32 units)
    long long last_injected;
    long long last_removed;
    double surface_field;       // E_s that produced n_inj
    unsigned int flags;         // SCLF_FLAG_* (sticky)
    unsigned int load_bad;      // set by the validation of loaded particles
    // accumulated by the particle kernel during a step
    unsigned long long acc_w0;
    unsigned long long acc_removed;
    long long inj_done;         // injections actually performed this step
    // compaction bookkeeping
    unsigned int ticket;        // tile ticket of the compaction kernel
    unsigned int compact_epoch; // tags tile states of one compaction
    unsigned long long slots_processed;  // running sum of slots pushed
    long long max_id;           // largest loaded particle ID
    long long pad1[2];
};

// Particles that leave a sub-domain's cell range for a neighbour's (z-domain
// decomposition of one tube): the particle kernel appends them here (one
// outbox per direction); the decomposed tube's exchange moves them into the
// neighbour's slots after the step. x holds positions in the tube's particle
// format (Real, or int32 for SCLF_FIX32).
struct Outbox {
    void* x;
    void* u;
    long long* ids;            // null when the tube keeps no IDs
    unsigned long long* n;     // count (atomically incremented); null: no outbox
    long long cap;
};

// Per-step event log of a recorded run: kLogStride entries per step, indexed
// by the step counter DevState::step.
constexpr int kLogStride = 4;
constexpr int kLogSlots = 0;     // slots before the step's injection
constexpr int kLogInjected = 1;  // electrons injected by the step
constexpr int kLogRemoved = 2;   // particles that left the tube (or went non-finite)

// Constants of one tube in the precision the kernels use.
struct FieldConsts {
    int nz;
    double dt, cdt, fourpi_dt, s_over_dt;
    double four_pi_s, two_pi_dz_rho0, sheet;
};

template <class Real>
struct PushArgs {
    DevState* st;
    Real* xi;                  // slot positions in cell units (hole: < 0)
    Real* u;                   // gamma beta
    Real* xo;                  // where the pushed slots go (xi itself: in place)
    Real* uo;
    long long* ids;            // may be null
    const Real* ez2;           // gather table, 2*(nz+1): (E_{m-1/2}, E_{m+1/2})
    long long* evlog;          // may be null: records slots and injections per step
    const long long* replay;   // may be null: injection counts to use instead
                               // of the tube's own (a log in the evlog layout)
    void* jacc;                // nz accumulators (long long or double)
    long long capacity;        // slots
    int nz;
    Real nzf;                  // (Real)nz
    Real dt;                   // (Real)dt
    Real cfl;                  // (Real)(dt/dz)
    // owned cells [lo, hi) of a sub-domain (0, nz for a whole tube): a particle
    // that ends inside the tube but outside them goes to out[0] (below) or
    // out[1] (above), a device array of two outboxes (null for a whole tube)
    int lo, hi;
    const Outbox* out;
};

template <class Real>
struct FieldArgs {
    DevState* st;
    double* ez;                // nz cells, E_z^n -> E_z^{n+1}
    const double* er_in;       // nz+1 nodes, E_r^n
    double* er_out;            // nz+1 nodes, E_r^{n+1}
    const double* b_in;        // nz cells, B^{n+1/2}
    double* b_out;             // nz cells, B^{n+3/2}
    void* jacc;                // nz accumulators, zeroed after use
    double* jlast;             // nz cells, J^{n+1/2} (diagnostic copy)
    Real* ez2;                 // gather table for the next step
    long long* evlog;          // may be null: records the step's removals
    FieldConsts c;
    int lo, hi;                // cells updated: [lo, hi) (0, nz for a whole tube)
};

// Particle kernel of the SCLF_FIX32 mode: positions X = xi 2^fb (int32,
// holes < 0), momenta float32, fixed-point current.
struct PushFixArgs {
    DevState* st;
    int* X;
    float* u;
    int* Xo;                   // where the pushed slots go (X itself: in place)
    float* uo;
    long long* ids;            // may be null
    const float* ez2;          // gather table, float32
    long long* evlog;          // may be null: records slots and injections per step
    const long long* replay;   // may be null: injection counts to use instead
    long long* jacc;           // nz accumulators, 2^-32 units
    long long capacity;
    int nz;
    int fb;                    // fractional bits
    float dt;                  // (float)dt
    float cfl;                 // (float)(dt/dz)
    float scale;               // 2^-fb
    float two_fb;              // 2^fb
    int lo, hi;                // owned cells (see PushArgs)
    const Outbox* out;
};

template <class Pos, class Mom>
struct CompactArgs {
    DevState* st;
    Pos* xi;                         // holes: xi < 0
    Mom* u;
    long long* ids;
    unsigned long long* tile_state;  // one word per tile
    long long capacity;
    int force;                       // 0: only when holes or capacity call for it
    int withhold_first;              // self-test: tile 0 publishes nothing, so the
                                     // look-back of tile 1 must give up
    long long spin_limit;            // polls of a look-back before it gives up
};
constexpr long long kCompactSpinLimit = 1LL << 22;   // x >= 64 ns: about a quarter second

// One tube of a batch, as the batched kernels see it (FP32 particles,
// fixed-point current).
struct alignas(128) BatchTube {
    // what the particle kernel reads, within one 128-byte line
    DevState* st;
    float* xi;
    float* u;
    long long* ids;
    float* ez2;                // gather table (read by the particle kernel, written by the field kernel)
    long long* jacc;
    long long tile0;           // first tile of this tube in the batch's tile space
    long long n_slots;         // this step: slots before the injection,
    long long n_tot;           //   slots after it (injection clipped to the capacity),
    long long id0;             //   first ID handed out,
    long long n_req;           //   injection requested (refreshed before each particle launch)
    int nz;
    float nzf, dt, cfl;
    // the rest
    long long capacity;
    int cell0;                 // first cell of this tube in the batch's cell space
    int fb;                    // SCLF_FIX32 batches: fractional bits of the positions (xi holds int32)
    double* ez;
    double* er[2];
    double* b[2];
    double* jlast;
    FieldConsts fc;
};

// Reverse sweep of one step (the discrete adjoint, adjoint.cu).
// The transposed field update of Eq. 3, one thread per cell: adjoints of
// (E_z, E_r, B) after the step -> before it, and of the current J.
template <class Real>
struct AdjFieldArgs {
    double* lez;               // nz cells, in place: after -> before the step
    const double* ler_in;      // nz+1 nodes, after the step
    double* ler_out;           // nz+1 nodes, before the step
    const double* lb_in;       // nz cells, after the step
    double* lb_out;            // nz cells, before the step
    const double* jstep;       // nz cells, J^{n+1/2} of the step (forward)
    double* lsum;              // nz cells: += lambda_J J (for d/ds)
    Real* ls_tab;              // nz cells: (s/dt) lambda_J, read by the particles
    int nz;
    double dt, cdt, fourpi_dt, s_over_dt;
};

// Per particle: adjoints of the deposit, the Eq. 1 push and the gather.
template <class Real>
struct AdjPushArgs {
    const Real* xi;            // slots before the step (holes < 0)
    const Real* u;
    Real* lx;                  // in: adjoint of the slots after the step;
    Real* lu;                  // out: before it (in place)
    const Real* ez2;           // the step's gather table
    const Real* ls_tab;        // (s/dt) lambda_J per cell
    double* lez;               // nz cells: the gather's share is added
    const long long* log;      // the step's kLogStride log entries
    unsigned int* flags;       // the tube's status word (bounds-checked builds)
    int nz;
    Real nzf, dt, cfl;
};

// The same for SCLF_FIX32 positions (X = xi 2^fb, holes < 0); adjoints in
// cell units, float32.
struct AdjPushFixArgs {
    const int* X;
    const float* u;
    float* lx;
    float* lu;
    const float* ez2;
    const float* ls_tab;
    double* lez;
    const long long* log;
    unsigned int* flags;       // the tube's status word (bounds-checked builds)
    int nz, fb;
    float dt, cfl, scale, two_fb;
};

// Launch of `kernel` on `grid` x `block` threads. With `overlap` the launch
// carries programmatic stream serialisation: the grid may be launched while
// the kernel before it in the stream is finishing (as that kernel's CTAs
// exit). Such a kernel begins with grid_dependency_wait(), which returns once
// that kernel has completed and its writes are visible, so the two kernels'
// memory accesses keep stream order; what overlaps is the launch. A preceding
// operation that is not a kernel (a copy, an event) is waited for in full.
template <class... P, class... A>
inline cudaError_t launch_kernel(void (*kernel)(P...), int grid, int block, size_t smem,
                                 cudaStream_t s, bool overlap, const A&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(block));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1u : 0u;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Launchers. All return the launch's error (cudaGetLastError() after <<<>>>).
// Those with `overlap` pass it to launch_kernel.
// The single-tube particle kernels take `stages`: 1 loads each tile straight
// into registers, 2..kMaxPushStages stream the next tiles through a ring of
// that many shared-memory stages by bulk asynchronous copies (TMA).
constexpr int kMaxPushStages = 4;
constexpr int kDefaultPushStages = 1;
template <class Real>
cudaError_t launch_push(const PushArgs<Real>& a, int accumulate, int stages, int grid,
                        cudaStream_t s, bool overlap = false);
template <class Real>
int push_grid_size(int accumulate, int stages, int device_sms);
template <class Real>
cudaError_t launch_field(const FieldArgs<Real>& a, int accumulate,
                         cudaStream_t s, bool overlap = false);
cudaError_t launch_push_fix32(const PushFixArgs& a, int stages, int grid, cudaStream_t s,
                              bool overlap = false);
// Shapes of the batched particle kernel: particles per thread (the tile is
// kThreads times that), CTAs per SM in its launch bounds and per-thread
// current runs (1: the first particle's cell; 2: also the last one's).
constexpr int kBatchVariants = 6;
constexpr int kBatchPPT[kBatchVariants] = {8, 8, 4, 8, 8, 16};
constexpr int kBatchMinBlocks[kBatchVariants] = {4, 3, 4, 4, 3, 2};
constexpr int kBatchRuns[kBatchVariants] = {1, 1, 1, 2, 2, 2};
cudaError_t launch_batch_push(const BatchTube* tubes, const int* tile_tube, long long n_tiles,
                              int grid, int variant, cudaStream_t s, bool overlap = false);
// A tube's constants for the batched particle kernel, passed by value in the
// kernel's parameter space (the constant bank, 32 KB at most): the compiler
// reloads them instead of holding them in registers across a tile. Batches
// of up to kBatchConstTubes tubes use it; larger ones read the descriptors.
struct BatchConst {
    DevState* st;
    float* xi;
    float* u;
    long long* ids;
    const float* ez2;
    long long* jacc;
    long long tile0;
    int nz;
    float nzf, dt, cfl;
};
constexpr int kBatchConstTubes = 400;
struct BatchConstTable {
    BatchConst t[kBatchConstTubes];
};
static_assert(sizeof(BatchConstTable) + 3 * sizeof(void*) <= 32764,
              "kernel parameters are limited to 32764 bytes");
cudaError_t launch_batch_push_const(const BatchConstTable& k, const BatchTube* tubes,
                                    const int* tile_tube, long long n_tiles, int grid,
                                    int variant, cudaStream_t s, bool overlap = false);
int batch_push_const_grid_size(int variant, int device_sms);
// Copies each tube's step counters (slots, clipped injection, first ID) into
// its descriptor before the particle launch.
cudaError_t launch_batch_refresh(BatchTube* tubes, int n_tubes, cudaStream_t s,
                                 bool overlap = false);
cudaError_t launch_batch_status(const BatchTube* tubes, int n_tubes, tube_stats* out,
                                cudaStream_t s);
int batch_push_grid_size(int variant, int device_sms);
cudaError_t launch_batch_field(const BatchTube* tubes, const int* cell_tube, int n_cells,
                               int parity, cudaStream_t s, bool overlap = false);
int push_fix32_grid_size(int stages, int device_sms);
// The SCLF_FIX32 batch's particle kernel (one shape: 8 slots per thread).
cudaError_t launch_batch_push_fix32(const BatchTube* tubes, const int* tile_tube,
                                    long long n_tiles, int grid, cudaStream_t s,
                                    bool overlap = false);
int batch_push_fix32_grid_size(int device_sms);
template <class Pos, class Mom>
cudaError_t launch_compact(const CompactArgs<Pos, Mom>& a, int grid, cudaStream_t s);
template <class Pos, class Mom>
int compact_grid_size(int device_sms);
template <class Pos, class Mom>
cudaError_t launch_append(DevState* st, Pos* xi, Mom* u, long long* ids,
                          long long first, long long n, bool zero_particles,
                          cudaStream_t s);
template <class Real>
cudaError_t launch_base_weight(DevState* st, const Real* xi, long long n_slots,
                               cudaStream_t s);
cudaError_t launch_base_weight_fix32(DevState* st, const int* X, long long n_slots,
                                     int fb, cudaStream_t s);
// Checks n loaded slots: 0 <= position < top (in stored position units, as a
// double so that Nz 2^fb = 2^31 fits), finite momentum, IDs >= 0
// (sets st->load_bad), and the largest ID (st->max_id).
template <class Pos, class Mom>
cudaError_t launch_validate(DevState* st, const Pos* xi, const Mom* u, const long long* ids,
                            long long n, double top, cudaStream_t s);
// Over the live slots [0, n): out[0] = count, out[1] = sum of gamma,
// out[2] = max gamma (part: 3 * kDiagBlocks doubles of scratch).
constexpr int kDiagBlocks = 128;
template <class Pos, class Mom>
cudaError_t launch_particle_diag(const Pos* xi, const Mom* u, long long n, double* part,
                                 double* out, cudaStream_t s);
cudaError_t launch_finish_append(DevState* st, const double* ez,
                                 long long n_added, FieldConsts c,
                                 cudaStream_t s);
template <class Real>
cudaError_t launch_ez_table(const double* ez, Real* ez2, int nz, cudaStream_t s);
cudaError_t launch_velocity_check(unsigned first, unsigned long long count,
                                  unsigned long long* out, int grid, cudaStream_t s);
template <class Pos>
cudaError_t launch_rho(const Pos* xi, long long n_slots, double* rho_acc,
                       int nz, double scale, cudaStream_t s);

template <class Real>
cudaError_t launch_adj_field(const AdjFieldArgs<Real>& a, cudaStream_t s, bool overlap = false);
template <class Real>
cudaError_t launch_adj_push(const AdjPushArgs<Real>& a, int grid, cudaStream_t s,
                            bool overlap = false);
template <class Real>
int adj_push_grid_size(int device_sms);
cudaError_t launch_adj_push_fix32(const AdjPushFixArgs& a, int grid, cudaStream_t s,
                                  bool overlap = false);
int adj_push_fix32_grid_size(int device_sms);
// Sums over the final state of a recorded run: out[0] = mean gamma of the
// live slots, out[1] = ||E_z||_2 = sqrt(sum E_z^2 dz). part holds
// 2 * kObjBlocks doubles.
constexpr int kObjBlocks = 256;
template <class Pos, class Mom>
cudaError_t launch_objectives(const Pos* xi, const Mom* u, const DevState* st,
                              const double* ez, int nz, double dz, double* part,
                              double* out, cudaStream_t s);
// Adjoint seeds: lambda_u = u / gamma / N_live (mean gamma), lambda_E =
// E dz / ||E|| (field norm).
template <class Pos, class Mom>
cudaError_t launch_seed_gamma(const Pos* xi, const Mom* u, const DevState* st, Mom* lx,
                              Mom* lu, cudaStream_t s);
cudaError_t launch_seed_ez(const double* ez, int nz, double dz, const double* values,
                           double* lez, cudaStream_t s);

// Stable sort of n slots by cell (sort.cu): keys = cell (holes: nz, last),
// LSD radix with 8-bit digits; xo/uo/io receive the permuted slots. scale
// converts a stored position to cells (2^-fb for SCLF_FIX32, else 1).
long long sort_scratch_bytes(long long n);
template <class Pos, class Mom>
cudaError_t launch_sort_by_cell(const Pos* xi, const Mom* u, const long long* ids, long long n,
                                int nz, double scale, void* scratch, Pos* xo, Mom* uo,
                                long long* io, cudaStream_t s);

// Host set-up (setup.cpp).
int derive(const tube_params* p, tube_derived* d);
int build_rho_gj(const tube_params* p, const tube_derived* d, double* rho);
void solve_poisson(const double* rho, int64_t nz, double dz, double* phi);
// Transpose of solve_poisson: from the adjoint of phi (nodes 0..Nz) to that
// of the source rho (nodes 0..Nz; node 0 gets 0).
void solve_poisson_transpose(const double* lphi, int64_t nz, double dz, double* lrho);
// grad[0..2] = d/d(B, P, R) of sum_j d_rho_j rho_GJ,j (grid, dt, s fixed).
int rho_gj_parameter_gradient(const tube_params* p, const double* d_rho, double* grad);

}  // namespace sclf
