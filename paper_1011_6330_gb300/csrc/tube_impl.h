// Internal definition of a tube (struct sclf_tube) and the helpers that the
// translation units driving tubes (the tube and batch ABI, the adjoint
// driver) share. Not part of the C ABI.
#pragma once

#include <cstdio>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sclf_internal.h"

namespace sclf {

// Byte offsets of the arrays in a tube's device workspace.
struct TubeLayout {
    int64_t cap_pad = 0, ntiles = 0;
    int64_t off_state = 0, off_xi = 0, off_u = 0, off_ids = 0, off_tiles = 0;
    int64_t off_ez = 0, off_er = 0, off_b = 0, off_jacc = 0, off_jlast = 0;
    int64_t off_ez2 = 0, off_rho = 0, off_diag = 0, total = 0;
};

}  // namespace sclf

struct sclf_tube {
    tube_params p{};
    tube_derived d{};
    sclf::TubeLayout lay;
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t gstream = nullptr;     // stream used for graph capture/replay
    bool own_gstream = false;
    bool owns_ws = false;
    char* ws = nullptr;
    sclf::DevState* st = nullptr;
    void* xi = nullptr;
    void* u = nullptr;
    long long* ids = nullptr;
    unsigned long long* tiles = nullptr;
    double* ez = nullptr;
    double* er[2] = {nullptr, nullptr};
    double* b[2] = {nullptr, nullptr};
    void* jacc = nullptr;
    double* jlast = nullptr;
    void* ez2 = nullptr;
    double* rho_acc = nullptr;
    double* diag = nullptr;            // scratch of tube_diagnostics
    std::vector<double> rho_gj;
    std::vector<double> gr_f, gr_H;     // copies of the caller's Eq. 6 tables (p points here)
    sclf::FieldConsts fc{};
    int push_grid = 0, compact_grid = 0;
    int push_stages = 1;               // the particle kernel's TMA ring (1: none)
    bool overlap = true;               // step kernels by programmatic dependent launch
    int fb = 0;                        // fractional bits of SCLF_FIX32 positions
    int64_t host_step = 0;             // steps launched (== device step count)
    int steps_since_compact = 0;
    int compact_every = 64;
    // graphs
    cudaGraphExec_t chunk = nullptr;
    int chunk_steps = 0;
    cudaEvent_t fork = nullptr, join = nullptr;
    // timed graphs: two copies with their own events, replayed alternately so
    // one can be read back while the other runs
    struct TimedChunk {
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> ev;   // 3 per step + 2 around the compaction
        bool pending = false;
    } tchunk[2];
    int tnext = 0;
    // timing
    bool timing = false;
    int timing_every = 1;              // sampling period (units of work)
    int64_t timing_tick = 0;
    std::vector<cudaEvent_t> ev;       // pool, 3 per step, 2 per compaction
    struct Rec { int kind; int e0; };  // kind 0 step (e0, e0+1, e0+2), 1 compaction
    std::vector<Rec> recs;
    int ev_next = 0;
    tube_timing acc{};
    unsigned long long slots_base = 0;
    char* sort_ws = nullptr;           // scratch of tube_sort (allocated on first use)
    int steps_since_sort = 0;
    bool owned = false;                // stepped by a batch or an adjoint driver,
                                       // not by tube_step / tube_run
    // tube_status_async: copies of the device counters in a pinned ring
    // (allocated on first use), slot = ticket mod kStatusRing
    static constexpr int64_t kStatusRing = 1024;
    sclf::DevState* status_ring = nullptr;
    int64_t status_next = 0;
    // sub-domain of a decomposed tube: owned cells [dom_lo, dom_hi) and the
    // outboxes of particles leaving them (a whole tube: 0, Nz, none)
    int dom_lo = 0, dom_hi = 0;
    sclf::Outbox out_down{}, out_up{};
    const sclf::Outbox* out_dev = nullptr;   // the two above, in device memory
};

namespace sclf {

// An NVTX range over a host entry point (visible to ncu --nvtx and to any
// timeline profiler; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

inline int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return SCLF_OK;
    std::fprintf(stderr, "sclf_tube: CUDA error %s\n", cudaGetErrorString(e));
    return SCLF_ECUDA;
}
#define CK(x) do { const cudaError_t _e = (x); if (_e != cudaSuccess) return cuda_fail(_e); } while (0)

inline bool fp64(const sclf_tube* t) { return t->p.precision == SCLF_FP64; }
inline bool fix32(const sclf_tube* t) { return t->p.precision == SCLF_FIX32; }

template <class Real>
inline PushArgs<Real> push_args(sclf_tube* t) {
    PushArgs<Real> a;
    a.st = t->st;
    a.xi = static_cast<Real*>(t->xi);
    a.u = static_cast<Real*>(t->u);
    a.xo = a.xi;
    a.uo = a.u;
    a.ids = t->ids;
    a.ez2 = static_cast<const Real*>(t->ez2);
    a.evlog = nullptr;
    a.replay = nullptr;
    a.jacc = t->jacc;
    a.capacity = t->p.capacity;
    a.nz = static_cast<int>(t->p.Nz);
    a.nzf = static_cast<Real>(t->p.Nz);
    a.dt = static_cast<Real>(t->d.dt);
    a.cfl = static_cast<Real>(t->d.dt / t->d.dz);
    a.lo = t->dom_lo;
    a.hi = t->dom_hi;
    a.out = t->out_dev;
    return a;
}

template <class Real>
inline FieldArgs<Real> field_args(sclf_tube* t, int parity) {
    FieldArgs<Real> a;
    a.st = t->st;
    a.ez = t->ez;
    a.er_in = t->er[parity];
    a.er_out = t->er[parity ^ 1];
    a.b_in = t->b[parity];
    a.b_out = t->b[parity ^ 1];
    a.jacc = t->jacc;
    a.jlast = t->jlast;
    a.ez2 = static_cast<Real*>(t->ez2);
    a.evlog = nullptr;
    a.c = t->fc;
    a.lo = t->dom_lo;
    a.hi = t->dom_hi;
    return a;
}

inline PushFixArgs push_fix_args(sclf_tube* t) {
    PushFixArgs a;
    a.st = t->st;
    a.X = static_cast<int*>(t->xi);
    a.u = static_cast<float*>(t->u);
    a.Xo = a.X;
    a.uo = a.u;
    a.ids = t->ids;
    a.ez2 = static_cast<const float*>(t->ez2);
    a.evlog = nullptr;
    a.replay = nullptr;
    a.jacc = static_cast<long long*>(t->jacc);
    a.capacity = t->p.capacity;
    a.nz = static_cast<int>(t->p.Nz);
    a.fb = t->fb;
    a.dt = static_cast<float>(t->d.dt);
    a.cfl = static_cast<float>(t->d.dt / t->d.dz);
    a.scale = std::ldexp(1.0f, -t->fb);
    a.two_fb = std::ldexp(1.0f, t->fb);
    a.lo = t->dom_lo;
    a.hi = t->dom_hi;
    a.out = t->out_dev;
    return a;
}

inline cudaError_t do_ez_table(sclf_tube* t) {
    const int nz = static_cast<int>(t->p.Nz);
    return fp64(t) ? launch_ez_table<double>(t->ez, static_cast<double*>(t->ez2), nz, t->stream)
                   : launch_ez_table<float>(t->ez, static_cast<float*>(t->ez2), nz, t->stream);
}

// Shared with the decomposed-tube driver (defined in tube.cu).
cudaError_t enqueue_push(sclf_tube* t, cudaStream_t s);
cudaError_t enqueue_field(sclf_tube* t, int parity, cudaStream_t s);
cudaError_t enqueue_compact(sclf_tube* t, cudaStream_t s, int force);
double raw_cells(const sclf_tube* t, const void* raw, int64_t i);
int append_raw(sclf_tube* t, int64_t n, const void* xi, const void* u, const int64_t* id);
int native_particles(const sclf_tube* t, int64_t n, const double* z, const double* u,
                     std::vector<char>& xs, std::vector<char>& us);
int set_fields_host(sclf_tube* t, const double* ez, const double* er, const double* b);

inline int read_state(sclf_tube* t, DevState* h) {
    CK(cudaMemcpyAsync(h, t->st, sizeof(DevState), cudaMemcpyDeviceToHost, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    return SCLF_OK;
}

}  // namespace sclf
