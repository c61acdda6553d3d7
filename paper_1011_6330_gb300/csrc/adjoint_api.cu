// C ABI of the adjoint driver (declared in include/sclf_tube.h). A tube's
// N-step run (Sec. 2, Figure A) is recorded with checkpoints every K steps
// and then swept in reverse segment by segment: each segment is recomputed
// from its checkpoint with its injection counts replayed, keeping every
// step's particle arrays, gather table and current, and the reverse kernels
// walk it back. The result is the gradient of an objective with respect to
// rho_GJ at the nodes and to the macro charge s; through rho_GJ's closed
// form (Eq. 5-7) it is chained to the pulsar's B, P and R.
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "tube_impl.h"

using namespace sclf;

struct sclf_adjoint {
    sclf_tube* t = nullptr;
    int64_t nsteps = 0;
    int K = 0;                      // steps per segment (even)
    int64_t nseg = 0;
    int64_t rs = 4;                 // bytes of one particle coordinate
    int64_t cap_pad = 0;
    int nz = 0;
    char* mem = nullptr;            // one device allocation for everything below
    std::vector<char*> sx, su;      // K+1 snapshots of the slot arrays of a segment
    char* ck_x = nullptr;           // nseg+1 checkpoints (segment starts and the end)
    char* ck_u = nullptr;
    double* ck_f = nullptr;         // per checkpoint: E_z (nz), E_r (nz+1), B (nz)
    DevState* ck_st = nullptr;      // per checkpoint
    char* tabs = nullptr;           // K+1 gather tables of a segment
    double* jlog = nullptr;         // K currents of a segment (nz each)
    long long* evlog = nullptr;     // kLogStride per step: the recorded events
    long long* ulog = nullptr;      // kLogStride per step: injections set by the caller
    long long* seglog = nullptr;    // kLogStride per step of the segment being reversed
    char* lx = nullptr;             // adjoints of the slots
    char* lu = nullptr;
    double* lez = nullptr;
    double* ler[2] = {nullptr, nullptr};
    double* lb[2] = {nullptr, nullptr};
    double* lsum = nullptr;         // per cell: sum over steps of lambda_J J
    char* ls_tab = nullptr;         // per cell: (s/dt) lambda_J in the particle precision
    double* part = nullptr;
    double* values = nullptr;       // the two objectives of the last forward pass
    double* weights = nullptr;      // nz cell weights of SCLF_OBJ_EZ_WEIGHTED
    bool have_weights = false;
    int adj_grid = 0;
    std::vector<double> rho_p0;     // particles' charge density at t = 0 (nodes)
    bool started = false;           // checkpoint 0 holds the initial state
    bool forward_done = false;
    bool use_ulog = false;
    int64_t current_seg = -1;       // segment whose steps the snapshots hold
    // Segment graphs of the four kinds (recorded forward, forward with the
    // caller's injections, recompute, reverse): one plain instance each and,
    // in timing mode, two instances with event-record nodes around every
    // kernel, replayed alternately so that one is read back while the other
    // runs.
    struct TimedGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> ev;   // 2K+1
        bool pending = false;
        int ka = 0, kb = 0;            // kernel kinds of its even and odd kernels
    };
    cudaGraphExec_t plain[4] = {nullptr, nullptr, nullptr, nullptr};
    TimedGraph timed[4][2];
    int tnext[4] = {0, 0, 0, 0};
    int timing = 0;                 // 0: off; n > 0: every n-th segment of a kind is timed
    int64_t seg_count[4] = {0, 0, 0, 0};
    double kms[6] = {0, 0, 0, 0, 0, 0};        // per kernel kind since timing was enabled
    int64_t klaunch[6] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    float fwd_ms = 0.f, bwd_ms = 0.f;
    int64_t pslots = 0;
};

namespace {

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

char* tab_of(sclf_adjoint* A, int k) {
    return A->tabs + static_cast<int64_t>(k) * align256(2 * (A->nz + 1) * A->rs);
}
double* ckf_of(sclf_adjoint* A, int64_t c) { return A->ck_f + c * (3 * A->nz + 1); }

// An event-record node of a timed segment graph (ev non-null): event 0 goes
// before the first kernel and events 2k+1, 2k+2 after the two kernels of
// the graph's k-th step.
cudaError_t mark(sclf_adjoint* A, const std::vector<cudaEvent_t>* ev, int i) {
    if (!ev) return cudaSuccess;
    return cudaEventRecordWithFlags((*ev)[i], A->t->gstream, cudaEventRecordExternal);
}

// K forward steps from snapshot 0: step k reads snapshot k and writes k+1.
// Pos is the stored position type (float, double, or int for SCLF_FIX32),
// Real the precision of the gather table and the particle adjoints.
template <class Pos, class Real>
int capture_forward(sclf_adjoint* A, long long* evlog, const long long* replay,
                    const std::vector<cudaEvent_t>* timed, cudaGraphExec_t* out) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = mark(A, timed, 0);
    for (int k = 0; k < A->K && e == cudaSuccess; ++k) {
        if constexpr (std::is_same<Pos, int>::value) {
            PushFixArgs pa = push_fix_args(t);
            pa.X = reinterpret_cast<int*>(A->sx[k]);
            pa.u = reinterpret_cast<float*>(A->su[k]);
            pa.Xo = reinterpret_cast<int*>(A->sx[k + 1]);
            pa.uo = reinterpret_cast<float*>(A->su[k + 1]);
            pa.ids = nullptr;
            pa.ez2 = reinterpret_cast<const float*>(tab_of(A, k));
            pa.evlog = evlog;
            pa.replay = replay;
            e = launch_push_fix32(pa, t->push_stages, t->push_grid, s, t->overlap);
        } else {
            PushArgs<Real> pa = push_args<Real>(t);
            pa.xi = reinterpret_cast<Real*>(A->sx[k]);
            pa.u = reinterpret_cast<Real*>(A->su[k]);
            pa.xo = reinterpret_cast<Real*>(A->sx[k + 1]);
            pa.uo = reinterpret_cast<Real*>(A->su[k + 1]);
            pa.ids = nullptr;
            pa.ez2 = reinterpret_cast<const Real*>(tab_of(A, k));
            pa.evlog = evlog;
            pa.replay = replay;
            e = launch_push<Real>(pa, t->p.accumulate, t->push_stages, t->push_grid, s,
                                  t->overlap);
        }
        if (e == cudaSuccess) e = mark(A, timed, 2 * k + 1);
        if (e != cudaSuccess) break;
        FieldArgs<Real> fa = field_args<Real>(t, k & 1);
        fa.jlast = A->jlog + static_cast<int64_t>(k) * A->nz;
        fa.ez2 = reinterpret_cast<Real*>(tab_of(A, k + 1));
        fa.evlog = evlog;
        e = launch_field<Real>(fa, t->p.accumulate, s, t->overlap);
        if (e == cudaSuccess) e = mark(A, timed, 2 * k + 2);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e); }
    CK(e2);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return SCLF_OK;
}

// The K steps of a segment in reverse: per step the transposed field update,
// then the particles.
template <class Pos, class Real>
int capture_reverse(sclf_adjoint* A, const std::vector<cudaEvent_t>* timed,
                    cudaGraphExec_t* out) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = mark(A, timed, 0);
    int i = 0;                       // reversed step index: events 2i, 2i+1, 2i+2
    for (int k = A->K - 1; k >= 0 && e == cudaSuccess; --k, ++i) {
        AdjFieldArgs<Real> fa;
        fa.lez = A->lez;
        fa.ler_in = A->ler[(k + 1) & 1];
        fa.ler_out = A->ler[k & 1];
        fa.lb_in = A->lb[(k + 1) & 1];
        fa.lb_out = A->lb[k & 1];
        fa.jstep = A->jlog + static_cast<int64_t>(k) * A->nz;
        fa.lsum = A->lsum;
        fa.ls_tab = reinterpret_cast<Real*>(A->ls_tab);
        fa.nz = A->nz;
        fa.dt = t->fc.dt;
        fa.cdt = t->fc.cdt;
        fa.fourpi_dt = t->fc.fourpi_dt;
        fa.s_over_dt = t->fc.s_over_dt;
        e = launch_adj_field<Real>(fa, s, t->overlap);
        if (e == cudaSuccess) e = mark(A, timed, 2 * i + 1);
        if (e != cudaSuccess) break;
        if constexpr (std::is_same<Pos, int>::value) {
            AdjPushFixArgs pa;
            pa.X = reinterpret_cast<const int*>(A->sx[k]);
            pa.u = reinterpret_cast<const float*>(A->su[k]);
            pa.lx = reinterpret_cast<float*>(A->lx);
            pa.lu = reinterpret_cast<float*>(A->lu);
            pa.ez2 = reinterpret_cast<const float*>(tab_of(A, k));
            pa.ls_tab = reinterpret_cast<const float*>(A->ls_tab);
            pa.lez = A->lez;
            pa.log = A->seglog + static_cast<int64_t>(kLogStride) * k;
            pa.flags = &t->st->flags;
            pa.nz = A->nz;
            pa.fb = t->fb;
            pa.dt = static_cast<float>(t->d.dt);
            pa.cfl = static_cast<float>(t->d.dt / t->d.dz);
            pa.scale = std::ldexp(1.0f, -t->fb);
            pa.two_fb = std::ldexp(1.0f, t->fb);
            e = launch_adj_push_fix32(pa, A->adj_grid, s, t->overlap);
        } else {
            AdjPushArgs<Real> pa;
            pa.xi = reinterpret_cast<const Real*>(A->sx[k]);
            pa.u = reinterpret_cast<const Real*>(A->su[k]);
            pa.lx = reinterpret_cast<Real*>(A->lx);
            pa.lu = reinterpret_cast<Real*>(A->lu);
            pa.ez2 = reinterpret_cast<const Real*>(tab_of(A, k));
            pa.ls_tab = reinterpret_cast<const Real*>(A->ls_tab);
            pa.lez = A->lez;
            pa.log = A->seglog + static_cast<int64_t>(kLogStride) * k;
            pa.flags = &t->st->flags;
            pa.nz = A->nz;
            pa.nzf = static_cast<Real>(A->nz);
            pa.dt = static_cast<Real>(t->d.dt);
            pa.cfl = static_cast<Real>(t->d.dt / t->d.dz);
            e = launch_adj_push<Real>(pa, A->adj_grid, s, t->overlap);
        }
        if (e == cudaSuccess) e = mark(A, timed, 2 * i + 2);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e); }
    CK(e2);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return SCLF_OK;
}

// Kernel kinds of the timing totals.
enum { kFwdPush, kFwdField, kRecPush, kRecField, kRevField, kRevPush };
// Segment graph kinds.
enum { kGraphFwd, kGraphFwdUser, kGraphRecompute, kGraphRev };

template <class Pos, class Real>
int capture_kind(sclf_adjoint* A, int kind, const std::vector<cudaEvent_t>* ev,
                 cudaGraphExec_t* out) {
    switch (kind) {
        case kGraphFwd: return capture_forward<Pos, Real>(A, A->evlog, nullptr, ev, out);
        case kGraphFwdUser: return capture_forward<Pos, Real>(A, A->evlog, A->ulog, ev, out);
        case kGraphRecompute: return capture_forward<Pos, Real>(A, nullptr, A->evlog, ev, out);
        default: return capture_reverse<Pos, Real>(A, ev, out);
    }
}

// Add a replayed timed graph's kernel durations to the totals (waits for it).
int collect(sclf_adjoint* A, sclf_adjoint::TimedGraph& g) {
    if (!g.pending) return SCLF_OK;
    CK(cudaEventSynchronize(g.ev[2 * A->K]));
    for (int k = 0; k < A->K; ++k) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, g.ev[2 * k], g.ev[2 * k + 1]));
        CK(cudaEventElapsedTime(&b, g.ev[2 * k + 1], g.ev[2 * k + 2]));
        A->kms[g.ka] += a;
        A->kms[g.kb] += b;
    }
    A->klaunch[g.ka] += A->K;
    A->klaunch[g.kb] += A->K;
    g.pending = false;
    return SCLF_OK;
}

int collect_all(sclf_adjoint* A) {
    for (auto& pair : A->timed)
        for (auto& g : pair) {
            const int rc = collect(A, g);
            if (rc) return rc;
        }
    return SCLF_OK;
}

// Launch one segment graph of the given kind (building it on first use). In
// timing mode every n-th segment of a kind replays a timed instance, after
// reading back the one replayed two timed launches ago.
template <class Pos, class Real>
int launch_segment(sclf_adjoint* A, int kind, int ka, int kb) {
    int rc;
    const bool timed = A->timing > 0 && A->seg_count[kind]++ % A->timing == 0;
    if (!timed) {
        if (!A->plain[kind] && (rc = capture_kind<Pos, Real>(A, kind, nullptr, &A->plain[kind])))
            return rc;
        CK(cudaGraphLaunch(A->plain[kind], A->t->gstream));
        return SCLF_OK;
    }
    auto& g = A->timed[kind][A->tnext[kind]];
    if (!g.exec) {
        g.ev.assign(2 * A->K + 1, nullptr);
        for (cudaEvent_t& e : g.ev)
            if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; return SCLF_ECUDA; }
        if ((rc = capture_kind<Pos, Real>(A, kind, &g.ev, &g.exec))) return rc;
    }
    if ((rc = collect(A, g))) return rc;
    CK(cudaGraphLaunch(g.exec, A->t->gstream));
    g.pending = true;
    g.ka = ka;
    g.kb = kb;
    A->tnext[kind] ^= 1;
    return SCLF_OK;
}

// Checkpoint c <- the state at a segment start (snapshot 0, fields at even
// parity, counters); and back.
int save_checkpoint(sclf_adjoint* A, int64_t c, int snap) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    const int64_t bytes = A->cap_pad * A->rs;
    const int64_t nz = A->nz;
    double* f = ckf_of(A, c);
    CK(cudaMemcpyAsync(A->ck_x + c * bytes, A->sx[snap], bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A->ck_u + c * bytes, A->su[snap], bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(f, t->ez, nz * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(f + nz, t->er[0], (nz + 1) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(f + 2 * nz + 1, t->b[0], nz * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A->ck_st + c, t->st, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
    return SCLF_OK;
}

int restore_fields(sclf_adjoint* A, int64_t c) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    const int64_t nz = A->nz;
    const double* f = ckf_of(A, c);
    CK(cudaMemcpyAsync(t->ez, f, nz * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->er[0], f + nz, (nz + 1) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->b[0], f + 2 * nz + 1, nz * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->st, A->ck_st + c, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
    return SCLF_OK;
}

int restore_checkpoint(sclf_adjoint* A, int64_t c) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    const int64_t bytes = A->cap_pad * A->rs;
    CK(cudaMemcpyAsync(A->sx[0], A->ck_x + c * bytes, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A->su[0], A->ck_u + c * bytes, bytes, cudaMemcpyDeviceToDevice, s));
    return restore_fields(A, c);
}

template <class Real>
cudaError_t table0(sclf_adjoint* A) {
    return launch_ez_table<Real>(A->t->ez, reinterpret_cast<Real*>(tab_of(A, 0)), A->nz,
                                 A->t->gstream);
}

template <class Pos, class Real>
int run_forward(sclf_adjoint* A, double* values) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    const int64_t nz = A->nz;
    const int64_t bytes = A->cap_pad * A->rs;
    int rc;
    if (!A->started) {
        // t = 0: Eq. 4 with the charge of the particles the tube holds
        A->rho_p0.assign(nz + 1, 0.0);
        rc = tube_read_fields(t, nullptr, nullptr, nullptr, nullptr, A->rho_p0.data());
        if (rc) return rc;
        rc = tube_solve_fields(t);
        if (rc) return rc;
        CK(cudaMemcpyAsync(A->sx[0], t->xi, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(A->su[0], t->u, bytes, cudaMemcpyDeviceToDevice, s));
        rc = save_checkpoint(A, 0, 0);
        if (rc) return rc;
        A->started = true;
    } else {
        rc = restore_checkpoint(A, 0);
        if (rc) return rc;
    }
    CK(table0<Real>(A));
    const int kind = A->use_ulog ? kGraphFwdUser : kGraphFwd;
    CK(cudaEventRecord(A->ev[0], s));
    for (int64_t c = 0; c < A->nseg; ++c) {
        if (c > 0) {
            rc = save_checkpoint(A, c, 0);
            if (rc) return rc;
        }
        rc = launch_segment<Pos, Real>(A, kind, kFwdPush, kFwdField);
        if (rc) return rc;
        if (c + 1 < A->nseg) {
            CK(cudaMemcpyAsync(A->sx[0], A->sx[A->K], bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(A->su[0], A->su[A->K], bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(tab_of(A, 0), tab_of(A, A->K), 2 * (nz + 1) * A->rs,
                               cudaMemcpyDeviceToDevice, s));
        }
    }
    CK(cudaEventRecord(A->ev[1], s));
    // the end of the run: checkpoint nseg, the objectives, the tube's own arrays
    rc = save_checkpoint(A, A->nseg, A->K);
    if (rc) return rc;
    CK((launch_objectives<Pos, Real>(reinterpret_cast<const Pos*>(A->sx[A->K]),
                                     reinterpret_cast<const Real*>(A->su[A->K]), t->st, t->ez,
                                     static_cast<int>(nz), t->d.dz, A->part, A->values, s)));
    CK(cudaMemcpyAsync(t->xi, A->sx[A->K], bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->u, A->su[A->K], bytes, cudaMemcpyDeviceToDevice, s));
    double hv[2];
    std::vector<long long> log(static_cast<size_t>(kLogStride * A->nsteps));
    CK(cudaMemcpyAsync(hv, A->values, sizeof(hv), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(log.data(), A->evlog, log.size() * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((rc = collect_all(A))) return rc;
    CK(cudaEventElapsedTime(&A->fwd_ms, A->ev[0], A->ev[1]));
    A->pslots = 0;
    for (int64_t n = 0; n < A->nsteps; ++n)
        A->pslots += log[kLogStride * n + kLogSlots] + log[kLogStride * n + kLogInjected];
    if (values) { values[0] = hv[0]; values[1] = hv[1]; }
    A->current_seg = A->nseg - 1;
    A->forward_done = true;
    return SCLF_OK;
}

template <class Pos, class Real>
int run_backward(sclf_adjoint* A, int objective, double* d_rho, double* d_s) {
    sclf_tube* t = A->t;
    cudaStream_t s = t->gstream;
    const int64_t nz = A->nz;
    const int64_t bytes = A->cap_pad * A->rs;
    int rc;
    // seeds at the end of the run (checkpoint nseg)
    CK(cudaMemsetAsync(A->lez, 0, nz * 8, s));
    CK(cudaMemsetAsync(A->ler[0], 0, (nz + 1) * 8, s));
    CK(cudaMemsetAsync(A->lb[0], 0, nz * 8, s));
    CK(cudaMemsetAsync(A->lsum, 0, nz * 8, s));
    CK(cudaMemsetAsync(A->lx, 0, bytes, s));
    CK(cudaMemsetAsync(A->lu, 0, bytes, s));
    if (objective == SCLF_OBJ_GAMMA) {
        CK((launch_seed_gamma<Pos, Real>(reinterpret_cast<const Pos*>(A->ck_x + A->nseg * bytes),
                                         reinterpret_cast<const Real*>(A->ck_u + A->nseg * bytes),
                                         A->ck_st + A->nseg, reinterpret_cast<Real*>(A->lx),
                                         reinterpret_cast<Real*>(A->lu), s)));
    } else if (objective == SCLF_OBJ_EZ) {
        CK(launch_seed_ez(ckf_of(A, A->nseg), static_cast<int>(nz), t->d.dz, A->values, A->lez, s));
    } else {                                      // d(sum_j w_j E_z,j)/dE_z = w
        CK(cudaMemcpyAsync(A->lez, A->weights, nz * 8, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaEventRecord(A->ev[2], s));
    for (int64_t c = A->nseg - 1; c >= 0; --c) {
        if (c != A->current_seg) {
            rc = restore_checkpoint(A, c);
            if (rc) return rc;
            CK(table0<Real>(A));
            rc = launch_segment<Pos, Real>(A, kGraphRecompute, kRecPush, kRecField);
            if (rc) return rc;
            A->current_seg = c;
        }
        CK(cudaMemcpyAsync(A->seglog, A->evlog + static_cast<int64_t>(kLogStride) * c * A->K,
                           static_cast<int64_t>(kLogStride) * A->K * 8, cudaMemcpyDeviceToDevice, s));
        rc = launch_segment<Pos, Real>(A, kGraphRev, kRevField, kRevPush);
        if (rc) return rc;
    }
    CK(cudaEventRecord(A->ev[3], s));
    // the tube shows the end of the run again
    rc = restore_fields(A, A->nseg);
    if (rc) return rc;
    std::vector<double> lez(nz), lphi(nz + 1), lsum(nz);
    CK(cudaMemcpyAsync(lez.data(), A->lez, nz * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(lphi.data(), A->ler[0], (nz + 1) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(lsum.data(), A->lsum, nz * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((rc = collect_all(A))) return rc;
    CK(cudaEventElapsedTime(&A->bwd_ms, A->ev[2], A->ev[3]));
    // t = 0: E_z = -(phi_{j+1} - phi_j)/dz, E_r = phi; phi from Eq. 4 with
    // source rho_GJ - rho_particles(s)
    const double dz = t->d.dz, sq = t->d.s;
    for (int64_t j = 0; j < nz; ++j) {
        lphi[j + 1] -= lez[j] / dz;
        lphi[j] += lez[j] / dz;
    }
    std::vector<double> lrho(nz + 1);
    solve_poisson_transpose(lphi.data(), nz, dz, lrho.data());
    double sj = 0.0, sp = 0.0;
    for (int64_t j = 0; j < nz; ++j) sj += lsum[j];
    for (int64_t j = 0; j <= nz; ++j) sp += lrho[j] * A->rho_p0[j];
    if (d_rho) std::memcpy(d_rho, lrho.data(), (nz + 1) * 8);
    if (d_s) *d_s = sj / sq - sp / sq;
    return SCLF_OK;
}

// Device bytes of a driver with segments of K steps (the allocation of
// adjoint_create, array by array).
int64_t adjoint_bytes(int64_t K, int64_t nsteps, int64_t nz, int64_t cap_pad, int64_t rs) {
    const int64_t bytes = cap_pad * rs, nseg = nsteps / K;
    return align256(2 * (K + 1) * bytes) + 2 * align256((nseg + 1) * bytes) +
           align256((nseg + 1) * (3 * nz + 1) * 8) +
           align256((nseg + 1) * static_cast<int64_t>(sizeof(DevState))) +
           align256((K + 1) * align256(2 * (nz + 1) * rs)) + align256(K * nz * 8) +
           2 * align256(kLogStride * nsteps * 8) + align256(kLogStride * K * 8) +
           2 * align256(bytes) + align256(nz * 8) + align256(2 * (nz + 1) * 8) +
           align256(2 * nz * 8) + align256(nz * 8) + align256(nz * rs) +
           align256(2 * kObjBlocks * 8) + align256(2 * 8) + align256(nz * 8);
}

void free_adjoint(sclf_adjoint* A) {
    if (!A) return;
    if (A->t) cudaStreamSynchronize(A->t->gstream);
    for (cudaGraphExec_t g : A->plain)
        if (g) cudaGraphExecDestroy(g);
    for (auto& pair : A->timed)
        for (auto& g : pair) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            for (cudaEvent_t e : g.ev)
                if (e) cudaEventDestroy(e);
        }
    for (cudaEvent_t e : A->ev)
        if (e) cudaEventDestroy(e);
    if (A->mem) cudaFree(A->mem);
    if (A->t) tube_destroy(A->t);
    delete A;
}

}  // namespace

extern "C" {

int adjoint_create(const tube_params* p, int64_t nsteps, int32_t checkpoint_every, void* stream,
                   adjoint_t* out) {
    if (!p || !out) return SCLF_EINVAL;
    *out = nullptr;
    if (p->precision != SCLF_FP32 && p->precision != SCLF_FP64 && p->precision != SCLF_FIX32)
        return SCLF_EINVAL;
    if (p->accumulate != SCLF_ACC_FIXED64) return SCLF_EINVAL;
    if (checkpoint_every < 0 || (checkpoint_every & 1) || nsteps <= 0 || (nsteps & 1) ||
        (checkpoint_every > 0 && nsteps % checkpoint_every != 0))
        return SCLF_EINVAL;
    tube_params q = *p;
    q.track_ids = 0;
    sclf_adjoint* A = new (std::nothrow) sclf_adjoint();
    if (!A) return SCLF_ENOMEM;
    int rc = tube_create(&q, nullptr, 0, stream, &A->t);
    if (rc) { delete A; return rc; }
    sclf_tube* t = A->t;
    t->owned = true;
    A->nsteps = nsteps;
    A->rs = p->precision == SCLF_FP64 ? 8 : 4;
    A->cap_pad = t->lay.cap_pad;
    A->nz = static_cast<int>(p->Nz);
    if (checkpoint_every == 0) {
        // the longest segment whose arrays fit in 80 % of the free device
        // memory: one segment (no recompute) when the whole run's snapshots fit
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { free_adjoint(A); return SCLF_ECUDA; }
        const double budget = 0.8 * static_cast<double>(free_b);
        int64_t best = 0;
        for (int64_t k = 2; k <= nsteps; k += 2)
            if (nsteps % k == 0 &&
                static_cast<double>(adjoint_bytes(k, nsteps, A->nz, A->cap_pad, A->rs)) <= budget)
                best = k;
        if (best == 0 || best > INT32_MAX) { free_adjoint(A); return SCLF_ENOMEM; }
        checkpoint_every = static_cast<int32_t>(best);
    }
    A->K = checkpoint_every;
    A->nseg = nsteps / checkpoint_every;
    const int64_t nz = A->nz, K = A->K, bytes = A->cap_pad * A->rs;
    // one allocation, every array 256-byte aligned (adjoint_bytes adds up the same)
    int64_t o = 0;
    auto take = [&](int64_t b) { const int64_t r = o; o += align256(b); return r; };
    const int64_t o_snap = take(2 * (K + 1) * bytes);
    const int64_t o_ckx = take((A->nseg + 1) * bytes);
    const int64_t o_cku = take((A->nseg + 1) * bytes);
    const int64_t o_ckf = take((A->nseg + 1) * (3 * nz + 1) * 8);
    const int64_t o_ckst = take((A->nseg + 1) * static_cast<int64_t>(sizeof(DevState)));
    const int64_t o_tabs = take((K + 1) * align256(2 * (nz + 1) * A->rs));
    const int64_t o_jlog = take(K * nz * 8);
    const int64_t o_evlog = take(kLogStride * nsteps * 8);
    const int64_t o_ulog = take(kLogStride * nsteps * 8);
    const int64_t o_seglog = take(kLogStride * K * 8);
    const int64_t o_lx = take(bytes);
    const int64_t o_lu = take(bytes);
    const int64_t o_lez = take(nz * 8);
    const int64_t o_ler = take(2 * (nz + 1) * 8);
    const int64_t o_lb = take(2 * nz * 8);
    const int64_t o_lsum = take(nz * 8);
    const int64_t o_lstab = take(nz * A->rs);
    const int64_t o_part = take(2 * kObjBlocks * 8);
    const int64_t o_values = take(2 * 8);
    const int64_t o_weights = take(nz * 8);
    if (cudaMalloc(&A->mem, o) != cudaSuccess) {
        A->mem = nullptr;
        free_adjoint(A);
        return SCLF_ENOMEM;
    }
    char* m = A->mem;
    for (int64_t k = 0; k <= K; ++k) {
        A->sx.push_back(m + o_snap + (2 * k) * bytes);
        A->su.push_back(m + o_snap + (2 * k + 1) * bytes);
    }
    A->ck_x = m + o_ckx;
    A->ck_u = m + o_cku;
    A->ck_f = reinterpret_cast<double*>(m + o_ckf);
    A->ck_st = reinterpret_cast<DevState*>(m + o_ckst);
    A->tabs = m + o_tabs;
    A->jlog = reinterpret_cast<double*>(m + o_jlog);
    A->evlog = reinterpret_cast<long long*>(m + o_evlog);
    A->ulog = reinterpret_cast<long long*>(m + o_ulog);
    A->seglog = reinterpret_cast<long long*>(m + o_seglog);
    A->lx = m + o_lx;
    A->lu = m + o_lu;
    A->lez = reinterpret_cast<double*>(m + o_lez);
    A->ler[0] = reinterpret_cast<double*>(m + o_ler);
    A->ler[1] = A->ler[0] + (nz + 1);
    A->lb[0] = reinterpret_cast<double*>(m + o_lb);
    A->lb[1] = A->lb[0] + nz;
    A->lsum = reinterpret_cast<double*>(m + o_lsum);
    A->ls_tab = m + o_lstab;
    A->part = reinterpret_cast<double*>(m + o_part);
    A->values = reinterpret_cast<double*>(m + o_values);
    A->weights = reinterpret_cast<double*>(m + o_weights);
    if (cudaMemsetAsync(A->mem, 0, o, t->gstream) != cudaSuccess ||
        cudaStreamSynchronize(t->gstream) != cudaSuccess) {
        free_adjoint(A);
        return SCLF_ECUDA;
    }
    for (cudaEvent_t& e : A->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; free_adjoint(A); return SCLF_ECUDA; }
    const int64_t tiles = A->cap_pad / (A->rs == 8 ? Layout<double>::kTile : Layout<float>::kTile);
    A->adj_grid = fix32(t) ? adj_push_fix32_grid_size(t->sms)
                : A->rs == 8 ? adj_push_grid_size<double>(t->sms) : adj_push_grid_size<float>(t->sms);
    if (A->adj_grid > tiles) A->adj_grid = static_cast<int>(tiles);
    *out = A;
    return SCLF_OK;
}

int adjoint_destroy(adjoint_t a) {
    if (!a) return SCLF_EINVAL;
    free_adjoint(a);
    return SCLF_OK;
}

int adjoint_checkpoint_every(adjoint_t a, int32_t* k) {
    if (!a || !k) return SCLF_EINVAL;
    *k = static_cast<int32_t>(a->K);
    return SCLF_OK;
}

int adjoint_tube(adjoint_t a, tube_t* out) {
    if (!a || !out) return SCLF_EINVAL;
    *out = a->t;
    return SCLF_OK;
}

int adjoint_set_injections(adjoint_t a, const int64_t* n_inj) {
    if (!a) return SCLF_EINVAL;
    if (!n_inj) {
        a->use_ulog = false;
        return SCLF_OK;
    }
    std::vector<long long> log(static_cast<size_t>(kLogStride * a->nsteps), 0);
    for (int64_t n = 0; n < a->nsteps; ++n) {
        if (n_inj[n] < 0) return SCLF_EINVAL;
        log[kLogStride * n + kLogInjected] = n_inj[n];
    }
    CK(cudaMemcpyAsync(a->ulog, log.data(), log.size() * 8, cudaMemcpyHostToDevice, a->t->gstream));
    CK(cudaStreamSynchronize(a->t->gstream));
    a->use_ulog = true;
    return SCLF_OK;
}

int adjoint_set_weights(adjoint_t a, const double* w) {
    if (!a || !w) return SCLF_EINVAL;
    for (int j = 0; j < a->nz; ++j)
        if (!std::isfinite(w[j])) return SCLF_EINVAL;
    CK(cudaMemcpyAsync(a->weights, w, static_cast<size_t>(a->nz) * 8, cudaMemcpyHostToDevice,
                       a->t->gstream));
    CK(cudaStreamSynchronize(a->t->gstream));
    a->have_weights = true;
    return SCLF_OK;
}

int adjoint_forward(adjoint_t a, double* values) {
    NvtxRange nvtx_range("adjoint_forward");
    if (!a) return SCLF_EINVAL;
    CK(cudaStreamSynchronize(a->t->stream));
    if (fix32(a->t)) return run_forward<int, float>(a, values);
    return a->rs == 8 ? run_forward<double, double>(a, values) : run_forward<float, float>(a, values);
}

int adjoint_events(adjoint_t a, int64_t* n_inj, int64_t* n_removed, int64_t* n_slots) {
    if (!a) return SCLF_EINVAL;
    if (!a->forward_done) return SCLF_ESTATE;
    std::vector<long long> log(static_cast<size_t>(kLogStride * a->nsteps));
    CK(cudaMemcpyAsync(log.data(), a->evlog, log.size() * 8, cudaMemcpyDeviceToHost, a->t->gstream));
    CK(cudaStreamSynchronize(a->t->gstream));
    for (int64_t n = 0; n < a->nsteps; ++n) {
        if (n_inj) n_inj[n] = log[kLogStride * n + kLogInjected];
        if (n_removed) n_removed[n] = log[kLogStride * n + kLogRemoved];
        if (n_slots) n_slots[n] = log[kLogStride * n + kLogSlots];
    }
    return SCLF_OK;
}

int adjoint_backward(adjoint_t a, int32_t objective, double* d_rho_gj, double* d_s) {
    NvtxRange nvtx_range("adjoint_backward");
    if (!a || (objective != SCLF_OBJ_GAMMA && objective != SCLF_OBJ_EZ &&
               objective != SCLF_OBJ_EZ_WEIGHTED))
        return SCLF_EINVAL;
    if (!a->forward_done || (objective == SCLF_OBJ_EZ_WEIGHTED && !a->have_weights))
        return SCLF_ESTATE;
    if (fix32(a->t)) return run_backward<int, float>(a, objective, d_rho_gj, d_s);
    return a->rs == 8 ? run_backward<double, double>(a, objective, d_rho_gj, d_s)
                      : run_backward<float, float>(a, objective, d_rho_gj, d_s);
}

int adjoint_param_gradient(adjoint_t a, const double* d_rho_gj, double d_s, double s_ref,
                           double* grad) {
    if (!a || !d_rho_gj || !grad || !std::isfinite(s_ref)) return SCLF_EINVAL;
    const int rc = rho_gj_parameter_gradient(&a->t->p, d_rho_gj, grad);
    if (rc) return rc;
    grad[3] = d_s * (s_ref != 0.0 ? s_ref : a->t->d.s);      // s = w s_ref
    return SCLF_OK;
}

int adjoint_timing(adjoint_t a, double* forward_ms, double* backward_ms, int64_t* particle_steps) {
    if (!a) return SCLF_EINVAL;
    if (forward_ms) *forward_ms = a->fwd_ms;
    if (backward_ms) *backward_ms = a->bwd_ms;
    if (particle_steps) *particle_steps = a->pslots;
    return SCLF_OK;
}

int adjoint_set_timing(adjoint_t a, int every) {
    if (!a || every < 0) return SCLF_EINVAL;
    CK(cudaStreamSynchronize(a->t->gstream));
    for (auto& pair : a->timed)
        for (auto& g : pair) g.pending = false;      // discard an earlier session
    a->timing = every;
    for (int64_t& c : a->seg_count) c = 0;
    for (int i = 0; i < 6; ++i) { a->kms[i] = 0.0; a->klaunch[i] = 0; }
    return SCLF_OK;
}

int adjoint_kernel_times(adjoint_t a, double* ms, int64_t* launches) {
    if (!a) return SCLF_EINVAL;
    for (int i = 0; i < 6; ++i) {
        if (ms) ms[i] = a->kms[i];
        if (launches) launches[i] = a->klaunch[i];
    }
    return SCLF_OK;
}

}  // extern "C"
