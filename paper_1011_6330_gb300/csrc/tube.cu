// C ABI of the sclf_tube library (declared in include/sclf_tube.h): tube
// creation, the step loop (direct launches or replayed CUDA graphs), device
// memory layout, read-back, checkpointing and event timing.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tube_impl.h"

using namespace sclf;

namespace {

constexpr double kPi = 3.14159265358979323846;

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

TubeLayout plan(const tube_params* p) {
    TubeLayout l;
    const int64_t rs = p->precision == SCLF_FP64 ? 8 : 4;
    const int64_t tile = p->precision == SCLF_FP64 ? Layout<double>::kTile : Layout<float>::kTile;
    const int64_t nz = p->Nz;
    l.cap_pad = align_up(p->capacity > 0 ? p->capacity : 1, kMaxTile);
    l.ntiles = l.cap_pad / tile;
    int64_t o = 0;
    auto take = [&](int64_t bytes) { const int64_t r = o; o = align_up(o + bytes, 256); return r; };
    l.off_state = take(sizeof(DevState));
    l.off_xi = take(l.cap_pad * rs);
    l.off_u = take(l.cap_pad * rs);
    l.off_ids = p->track_ids ? take(l.cap_pad * 8) : -1;
    l.off_tiles = take(l.ntiles * 8);
    l.off_ez = take(nz * 8);
    l.off_er = take(2 * (nz + 1) * 8);
    l.off_b = take(2 * nz * 8);
    l.off_jacc = take(nz * 8);
    l.off_jlast = take(nz * 8);
    l.off_ez2 = take(2 * (nz + 1) * rs);
    l.off_rho = take((nz + 1) * 8);
    l.off_diag = take((3 * kDiagBlocks + 4) * 8);
    l.total = o;
    return l;
}

}  // namespace


namespace {




template <class Pos, class Mom>
CompactArgs<Pos, Mom> compact_args(sclf_tube* t, int force) {
    CompactArgs<Pos, Mom> a;
    a.force = force;
    a.withhold_first = 0;
    a.spin_limit = kCompactSpinLimit;
    a.st = t->st;
    a.xi = static_cast<Pos*>(t->xi);
    a.u = static_cast<Mom*>(t->u);
    a.ids = t->ids;
    a.tile_state = t->tiles;
    a.capacity = t->p.capacity;
    return a;
}



// Per-precision launches of the small kernels.
cudaError_t do_append(sclf_tube* t, long long first, long long n, bool zero) {
    if (fp64(t))
        return launch_append<double, double>(t->st, static_cast<double*>(t->xi),
                                             static_cast<double*>(t->u), t->ids, first, n, zero, t->stream);
    if (fix32(t))
        return launch_append<int, float>(t->st, static_cast<int*>(t->xi), static_cast<float*>(t->u),
                                         t->ids, first, n, zero, t->stream);
    return launch_append<float, float>(t->st, static_cast<float*>(t->xi), static_cast<float*>(t->u),
                                       t->ids, first, n, zero, t->stream);
}
// Adds the base-cell weight of slots [first, first + n) to the accumulator
// that the next finish_append folds into W_0.
cudaError_t do_base_weight(sclf_tube* t, long long first, long long n) {
    if (fp64(t))
        return launch_base_weight<double>(t->st, static_cast<const double*>(t->xi) + first, n, t->stream);
    if (fix32(t))
        return launch_base_weight_fix32(t->st, static_cast<const int*>(t->xi) + first, n, t->fb, t->stream);
    return launch_base_weight<float>(t->st, static_cast<const float*>(t->xi) + first, n, t->stream);
}
cudaError_t do_rho(sclf_tube* t, long long slots) {
    const int nz = static_cast<int>(t->p.Nz);
    if (fp64(t)) return launch_rho<double>(static_cast<const double*>(t->xi), slots, t->rho_acc, nz, 1.0, t->stream);
    if (fix32(t)) return launch_rho<int>(static_cast<const int*>(t->xi), slots, t->rho_acc, nz,
                                         std::ldexp(1.0, -t->fb), t->stream);
    return launch_rho<float>(static_cast<const float*>(t->xi), slots, t->rho_acc, nz, 1.0, t->stream);
}
}  // namespace

namespace sclf {

// Position of raw slot i in cell units; negative for a hole.
double raw_cells(const sclf_tube* t, const void* raw, int64_t i) {
    if (fp64(t)) return static_cast<const double*>(raw)[i];
    if (fix32(t)) {
        const int X = static_cast<const int*>(raw)[i];
        return X < 0 ? -1.0 : std::ldexp(static_cast<double>(X), -t->fb);
    }
    return static_cast<const float*>(raw)[i];
}
double raw_mom(const sclf_tube* t, const void* raw, int64_t i) {
    return fp64(t) ? static_cast<const double*>(raw)[i] : double(static_cast<const float*>(raw)[i]);
}

cudaError_t enqueue_push(sclf_tube* t, cudaStream_t s) {
    if (fix32(t))
        return launch_push_fix32(push_fix_args(t), t->push_stages, t->push_grid, s, t->overlap);
    return fp64(t) ? launch_push<double>(push_args<double>(t), t->p.accumulate, t->push_stages,
                                         t->push_grid, s, t->overlap)
                   : launch_push<float>(push_args<float>(t), t->p.accumulate, t->push_stages,
                                        t->push_grid, s, t->overlap);
}
cudaError_t enqueue_field(sclf_tube* t, int parity, cudaStream_t s) {
    return fp64(t) ? launch_field<double>(field_args<double>(t, parity), t->p.accumulate, s,
                                          t->overlap)
                   : launch_field<float>(field_args<float>(t, parity), t->p.accumulate, s,
                                         t->overlap);
}
// The compaction follows a field kernel, whose commit resets the tile
// ticket; a compaction outside the step sequence resets it first.
cudaError_t enqueue_compact(sclf_tube* t, cudaStream_t s, int force) {
    if (force) {
        const cudaError_t e = cudaMemsetAsync(&t->st->ticket, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    if (fix32(t)) return launch_compact<int, float>(compact_args<int, float>(t, force), t->compact_grid, s);
    return fp64(t) ? launch_compact<double, double>(compact_args<double, double>(t, force), t->compact_grid, s)
                   : launch_compact<float, float>(compact_args<float, float>(t, force), t->compact_grid, s);
}


}  // namespace sclf

namespace {

int drain_timing(sclf_tube* t);

// Reserve k consecutive events of the timing pool; returns the first index
// or -1. Drains (synchronises) when the pool is full.
int reserve_events(sclf_tube* t, int k) {
    if (t->ev_next + k > static_cast<int>(t->ev.size())) {
        if (drain_timing(t) != SCLF_OK) return -1;
    }
    if (t->ev_next + k > static_cast<int>(t->ev.size())) return -1;
    const int e0 = t->ev_next;
    t->ev_next += k;
    return e0;
}

int one_step(sclf_tube* t) {
    const int parity = static_cast<int>(t->host_step & 1);
    const bool timed = t->timing && (t->timing_tick++ % t->timing_every) == 0;
    if (timed) {
        const int e0 = reserve_events(t, 3);
        if (e0 < 0) return SCLF_ECUDA;
        CK(cudaEventRecord(t->ev[e0], t->stream));
        CK(enqueue_push(t, t->stream));
        CK(cudaEventRecord(t->ev[e0 + 1], t->stream));
        CK(enqueue_field(t, parity, t->stream));
        CK(cudaEventRecord(t->ev[e0 + 2], t->stream));
        t->recs.push_back({0, e0});
    } else {
        CK(enqueue_push(t, t->stream));
        CK(enqueue_field(t, parity, t->stream));
    }
    t->host_step += 1;
    t->steps_since_compact += 1;
    if (t->timing) t->acc.steps_run += 1;
    if (t->steps_since_compact >= t->compact_every) {
        if (t->timing) t->acc.compactions_run += 1;
        if (t->timing) {
            const int e0 = reserve_events(t, 2);
            if (e0 < 0) return SCLF_ECUDA;
            CK(cudaEventRecord(t->ev[e0], t->stream));
            CK(enqueue_compact(t, t->stream, 0));
            CK(cudaEventRecord(t->ev[e0 + 1], t->stream));
            t->recs.push_back({1, e0});
        } else {
            CK(enqueue_compact(t, t->stream, 0));
        }
        t->steps_since_compact = 0;
    }
    return SCLF_OK;
}

// One captured graph = chunk_steps steps starting at even parity, then a
// compaction check (chunk_steps == compact interval, rounded up to even).
// With ev != nullptr, an event-record node precedes every kernel: ev[2k]
// step k's particle kernel, ev[2k+1] its field kernel, ev[2n] the
// compaction, and ev[2n+1] follows it (step k's field kernel ends at
// ev[2k+2]).
int capture_chunk(sclf_tube* t, cudaGraphExec_t* out, const std::vector<cudaEvent_t>* ev) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(t->gstream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    auto mark = [&](int i) {
        if (ev && e == cudaSuccess)
            e = cudaEventRecordWithFlags((*ev)[i], t->gstream, cudaEventRecordExternal);
    };
    const int n = t->chunk_steps;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        mark(2 * k);
        if (e == cudaSuccess) e = enqueue_push(t, t->gstream);
        mark(2 * k + 1);
        if (e == cudaSuccess) e = enqueue_field(t, k & 1, t->gstream);
    }
    mark(2 * n);
    if (e == cudaSuccess) e = enqueue_compact(t, t->gstream, 0);
    mark(2 * n + 1);
    const cudaError_t e2 = cudaStreamEndCapture(t->gstream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e); }
    CK(e2);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return SCLF_OK;
}

int build_chunk(sclf_tube* t) {
    if (t->chunk) return SCLF_OK;
    return capture_chunk(t, &t->chunk, nullptr);
}

// Add a replayed timed chunk's kernel times to the totals (waits for it).
int collect_chunk(sclf_tube* t, int which) {
    auto& c = t->tchunk[which];
    if (!c.pending) return SCLF_OK;
    const int n = t->chunk_steps;
    CK(cudaEventSynchronize(c.ev[2 * n + 1]));
    for (int k = 0; k < n; ++k) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, c.ev[2 * k], c.ev[2 * k + 1]));
        CK(cudaEventElapsedTime(&b, c.ev[2 * k + 1], c.ev[2 * k + 2]));
        t->acc.push_ms += a;
        t->acc.field_ms += b;
    }
    float cm = 0.f;
    CK(cudaEventElapsedTime(&cm, c.ev[2 * n], c.ev[2 * n + 1]));
    t->acc.compact_ms += cm;
    t->acc.n_compactions += 1;
    t->acc.n_steps += n;
    c.pending = false;
    return SCLF_OK;
}

int launch_graph(sclf_tube* t, cudaGraphExec_t exec) {
    if (t->gstream != t->stream) {
        CK(cudaEventRecord(t->fork, t->stream));
        CK(cudaStreamWaitEvent(t->gstream, t->fork, 0));
    }
    CK(cudaGraphLaunch(exec, t->gstream));
    if (t->gstream != t->stream) {
        CK(cudaEventRecord(t->join, t->gstream));
        CK(cudaStreamWaitEvent(t->stream, t->join, 0));
    }
    t->host_step += t->chunk_steps;
    t->steps_since_compact = 0;
    return SCLF_OK;
}

int launch_timed_chunk(sclf_tube* t) {
    const int w = t->tnext;
    auto& c = t->tchunk[w];
    int rc = collect_chunk(t, w);
    if (rc) return rc;
    if (!c.exec) {
        c.ev.resize(2 * t->chunk_steps + 2, nullptr);
        for (auto& e : c.ev) CK(cudaEventCreate(&e));
        rc = capture_chunk(t, &c.exec, &c.ev);
        if (rc) return rc;
    }
    rc = launch_graph(t, c.exec);
    if (rc) return rc;
    c.pending = true;
    t->tnext ^= 1;
    return SCLF_OK;
}

int launch_chunk(sclf_tube* t) { return launch_graph(t, t->chunk); }

int drain_timing(sclf_tube* t) {
    for (int w = 0; w < 2; ++w) {
        const int rc = collect_chunk(t, w);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(t->stream));
    for (const auto& r : t->recs) {
        float ms = 0.f;
        if (r.kind == 0) {
            CK(cudaEventElapsedTime(&ms, t->ev[r.e0], t->ev[r.e0 + 1]));
            t->acc.push_ms += ms;
            CK(cudaEventElapsedTime(&ms, t->ev[r.e0 + 1], t->ev[r.e0 + 2]));
            t->acc.field_ms += ms;
            t->acc.n_steps += 1;
        } else {
            CK(cudaEventElapsedTime(&ms, t->ev[r.e0], t->ev[r.e0 + 1]));
            t->acc.compact_ms += ms;
            t->acc.n_compactions += 1;
        }
    }
    t->recs.clear();
    t->ev_next = 0;
    return SCLF_OK;
}

template <class Real>
void to_native(const double* z, const double* u, int64_t n, double dz, std::vector<char>& xs,
               std::vector<char>& us) {
    xs.resize(n * sizeof(Real));
    us.resize(n * sizeof(Real));
    Real* x = reinterpret_cast<Real*>(xs.data());
    Real* v = reinterpret_cast<Real*>(us.data());
    for (int64_t i = 0; i < n; ++i) {
        x[i] = static_cast<Real>(z[i] / dz);
        v[i] = static_cast<Real>(u[i]);
    }
}

}  // namespace

namespace sclf {

// Append n raw particles (already in the tube's precision) after the slots.
int append_raw(sclf_tube* t, int64_t n, const void* xi, const void* u, const int64_t* id) {
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    if (h.n_slots + n > t->p.capacity) return SCLF_ECAPACITY;
    const int64_t rs = fp64(t) ? 8 : 4;
    if (n > 0) {
        CK(cudaMemcpyAsync(static_cast<char*>(t->xi) + h.n_slots * rs, xi, n * rs,
                           cudaMemcpyHostToDevice, t->stream));
        CK(cudaMemcpyAsync(static_cast<char*>(t->u) + h.n_slots * rs, u, n * rs,
                           cudaMemcpyHostToDevice, t->stream));
        if (t->ids) {
            if (id) {
                CK(cudaMemcpyAsync(t->ids + h.n_slots, id, n * 8, cudaMemcpyHostToDevice, t->stream));
            } else {
                CK(do_append(t, h.n_slots, n, false));
            }
        }
    }
    // W_0 is a sum over particles: add the new ones' share
    CK(do_base_weight(t, h.n_slots, n));
    CK(launch_finish_append(t->st, t->ez, n, t->fc, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    return SCLF_OK;
}

// Checks physical heights z in [0, L) and finite u, and converts them to the
// tube's raw particle format (cell units; FIX32: round-half-even(z/dz 2^fb)).
int native_particles(const sclf_tube* t, int64_t n, const double* z, const double* u,
                     std::vector<char>& xs, std::vector<char>& us) {
    for (int64_t i = 0; i < n; ++i)
        if (!(z[i] >= 0.0 && z[i] < t->d.L) || !std::isfinite(u[i])) return SCLF_EINVAL;
    if (fp64(t)) {
        to_native<double>(z, u, n, t->d.dz, xs, us);
    } else if (fix32(t)) {
        to_native<float>(z, u, n, t->d.dz, xs, us);
        int* X = reinterpret_cast<int*>(xs.data());
        const double top = std::ldexp(double(t->p.Nz), t->fb);
        for (int64_t i = 0; i < n; ++i) {
            const double v = std::nearbyint(std::ldexp(z[i] / t->d.dz, t->fb));
            if (!(v < top)) return SCLF_EINVAL;
            X[i] = static_cast<int>(v);
        }
    } else {
        to_native<float>(z, u, n, t->d.dz, xs, us);
    }
    // a position that rounds up to the top node is outside the tube
    for (int64_t i = 0; i < n; ++i)
        if (!(raw_cells(t, xs.data(), i) < double(t->p.Nz))) return SCLF_EINVAL;
    return SCLF_OK;
}

// Host fields (E_z at the Nz cells, E_r at the Nz+1 nodes, B_phi at the cells)
// into the tube's current copies, with the gather table, W_0 and the next
// injection count brought up to date.
int set_fields_host(sclf_tube* t, const double* ez, const double* er, const double* b) {
    const int64_t nz = t->p.Nz;
    const int par = static_cast<int>(t->host_step & 1);
    CK(cudaMemcpyAsync(t->ez, ez, nz * 8, cudaMemcpyHostToDevice, t->stream));
    CK(cudaMemcpyAsync(t->er[par], er, (nz + 1) * 8, cudaMemcpyHostToDevice, t->stream));
    if (b) CK(cudaMemcpyAsync(t->b[par], b, nz * 8, cudaMemcpyHostToDevice, t->stream));
    else CK(cudaMemsetAsync(t->b[par], 0, nz * 8, t->stream));
    CK(do_ez_table(t));
    DevState h;
    const int rc = read_state(t, &h);
    if (rc) return rc;
    CK(cudaMemsetAsync(&t->st->w0, 0, sizeof(long long), t->stream));
    CK(do_base_weight(t, 0, h.n_slots));
    CK(launch_finish_append(t->st, t->ez, 0, t->fc, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    return SCLF_OK;
}

}  // namespace sclf

namespace {

// The public view of the device counters.
void stats_from_state(const DevState& h, tube_stats* out) {
    out->step = h.step;
    out->n_particles = h.n_live;
    out->n_slots = h.n_slots;
    out->total_injected = h.total_injected;
    out->last_injected = h.last_injected;
    out->last_removed = h.last_removed;
    out->pending_injection = h.n_inj;
    out->surface_field = h.surface_field;
    out->flags = h.flags;
    out->reserved = 0;
}

}  // namespace

extern "C" {

int tube_params_default(tube_params* p) {
    if (!p) return SCLF_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->B_G = 1e12;
    p->P_s = 1.0;
    p->Rstar_cm = 1e6;
    p->incl_rad = 0.0;
    p->mass_g = 1.4 * 1.98847e33;
    p->R_cm = 0.0;
    p->L_over_R = 8.0;
    p->Nz = 1024;
    p->dt = 0.0;
    p->rho_gj_mode = SCLF_RHO_FLAT;
    p->precision = SCLF_FP32;
    p->macro_charge = 0.0;
    p->target_particles = 50000;
    p->capacity = 1 << 20;
    p->accumulate = SCLF_ACC_FIXED64;
    p->track_ids = 1;
    p->compact_interval = 64;
    p->use_graphs = 1;
    return SCLF_OK;
}

int tube_derive(const tube_params* p, tube_derived* d) { return derive(p, d); }

int tube_rho_gj_profile(const tube_params* p, double* rho) {
    if (!p || !rho) return SCLF_EINVAL;
    tube_derived d;
    const int rc = derive(p, &d);
    if (rc) return rc;
    return build_rho_gj(p, &d, rho);
}

int tube_rho_gj_param_gradient(const tube_params* p, const double* d_rho, double* grad) {
    if (!p || !d_rho || !grad) return SCLF_EINVAL;
    return rho_gj_parameter_gradient(p, d_rho, grad);
}

int tube_workspace_bytes(const tube_params* p, int64_t* bytes) {
    if (!p || !bytes) return SCLF_EINVAL;
    tube_derived d;
    const int rc = derive(p, &d);
    if (rc) return rc;
    *bytes = plan(p).total;
    return SCLF_OK;
}

int tube_create(const tube_params* p, void* dev_workspace, int64_t ws_bytes, void* stream,
                tube_t* out) {
    if (!p || !out) return SCLF_EINVAL;
    *out = nullptr;
    sclf_tube* t = new (std::nothrow) sclf_tube();
    if (!t) return SCLF_ENOMEM;
    t->p = *p;
    t->p.rho_gj_user = nullptr;
    int rc = derive(p, &t->d);
    if (rc) { delete t; return rc; }
    // the Eq. 6 tables stay with the tube (the adjoint's parameter chain reads them)
    if (p->rho_gj_mode == SCLF_RHO_GR && p->gr_f) t->gr_f.assign(p->gr_f, p->gr_f + p->Nz + 1);
    if (p->rho_gj_mode == SCLF_RHO_GR && p->gr_H) t->gr_H.assign(p->gr_H, p->gr_H + p->Nz + 1);
    t->p.gr_f = t->gr_f.empty() ? nullptr : t->gr_f.data();
    t->p.gr_H = t->gr_H.empty() ? nullptr : t->gr_H.data();
    t->lay = plan(p);
    t->fb = p->precision == SCLF_FIX32 ? fix32_bits(p->Nz) : 0;
    t->dom_lo = 0;                                   // the whole tube
    t->dom_hi = static_cast<int>(p->Nz);
    t->stream = static_cast<cudaStream_t>(stream);
    t->compact_every = p->compact_interval > 0 ? p->compact_interval : 64;
    t->chunk_steps = t->compact_every + (t->compact_every & 1);

    auto fail = [&](int code) { tube_destroy(t); return code; };
    if (cudaGetDevice(&t->device) != cudaSuccess) return fail(SCLF_ECUDA);
    if (cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess)
        return fail(SCLF_ECUDA);

    if (dev_workspace) {
        if (ws_bytes < t->lay.total || (reinterpret_cast<uintptr_t>(dev_workspace) & 255u))
            return fail(SCLF_ENOMEM);
        t->ws = static_cast<char*>(dev_workspace);
    } else {
        if (cudaMalloc(&t->ws, t->lay.total) != cudaSuccess) { t->ws = nullptr; return fail(SCLF_ENOMEM); }
        t->owns_ws = true;
    }
    const TubeLayout& l = t->lay;
    t->st = reinterpret_cast<DevState*>(t->ws + l.off_state);
    t->xi = t->ws + l.off_xi;
    t->u = t->ws + l.off_u;
    t->ids = l.off_ids >= 0 ? reinterpret_cast<long long*>(t->ws + l.off_ids) : nullptr;
    t->tiles = reinterpret_cast<unsigned long long*>(t->ws + l.off_tiles);
    t->ez = reinterpret_cast<double*>(t->ws + l.off_ez);
    t->er[0] = reinterpret_cast<double*>(t->ws + l.off_er);
    t->er[1] = t->er[0] + (p->Nz + 1);
    t->b[0] = reinterpret_cast<double*>(t->ws + l.off_b);
    t->b[1] = t->b[0] + p->Nz;
    t->jacc = t->ws + l.off_jacc;
    t->jlast = reinterpret_cast<double*>(t->ws + l.off_jlast);
    t->ez2 = t->ws + l.off_ez2;
    t->rho_acc = reinterpret_cast<double*>(t->ws + l.off_rho);
    t->diag = reinterpret_cast<double*>(t->ws + l.off_diag);

    // (a7) rho_GJ, Eq. 4 and the initial fields
    const int64_t nz = p->Nz;
    t->rho_gj.assign(nz + 1, 0.0);
    rc = build_rho_gj(p, &t->d, t->rho_gj.data());
    if (rc) return fail(rc);
    std::vector<double> phi(nz + 1), ez0(nz);
    solve_poisson(t->rho_gj.data(), nz, t->d.dz, phi.data());
    for (int64_t j = 0; j < nz; ++j) ez0[j] = -(phi[j + 1] - phi[j]) / t->d.dz;   // E_z = -phi'
    // E_r = phi / R with R = 1 (d/dr -> 1/R, phi = 0 on the wall)

    const double dt = t->d.dt, dz = t->d.dz, s = t->d.s;
    t->fc.nz = static_cast<int>(nz);
    t->fc.dt = dt;
    t->fc.cdt = dt / dz;
    t->fc.fourpi_dt = 4.0 * kPi * dt;
    t->fc.s_over_dt = s / dt;
    t->fc.four_pi_s = 4.0 * kPi * s;
    t->fc.two_pi_dz_rho0 = 2.0 * kPi * dz * t->rho_gj[0];
    t->fc.sheet = 4.0 * kPi * std::fabs(s);

    if (cudaMemsetAsync(t->ws, 0, l.total, t->stream) != cudaSuccess) return fail(SCLF_ECUDA);
    DevState h;
    std::memset(&h, 0, sizeof(h));
    h.compact_epoch = 1;
    if (cudaMemcpyAsync(t->st, &h, sizeof(h), cudaMemcpyHostToDevice, t->stream) ||
        cudaMemcpyAsync(t->ez, ez0.data(), nz * 8, cudaMemcpyHostToDevice, t->stream) ||
        cudaMemcpyAsync(t->er[0], phi.data(), (nz + 1) * 8, cudaMemcpyHostToDevice, t->stream))
        return fail(SCLF_ECUDA);
    cudaError_t e = do_ez_table(t);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    if (launch_finish_append(t->st, t->ez, 0, t->fc, t->stream) != cudaSuccess) return fail(SCLF_ECUDA);
    if (cudaStreamSynchronize(t->stream) != cudaSuccess) return fail(SCLF_ECUDA);

    t->push_stages = p->push_stages > 0 ? p->push_stages : kDefaultPushStages;
    t->overlap = p->launch_overlap >= 0;
    t->push_grid = fix32(t) ? push_fix32_grid_size(t->push_stages, t->sms)
                 : fp64(t) ? push_grid_size<double>(p->accumulate, t->push_stages, t->sms)
                           : push_grid_size<float>(p->accumulate, t->push_stages, t->sms);
    t->compact_grid = fix32(t) ? compact_grid_size<int, float>(t->sms)
                    : fp64(t) ? compact_grid_size<double, double>(t->sms)
                              : compact_grid_size<float, float>(t->sms);
    const int64_t tile = fp64(t) ? Layout<double>::kTile : Layout<float>::kTile;
    const int64_t max_tiles = l.cap_pad / tile;
    if (t->push_grid > max_tiles) t->push_grid = static_cast<int>(max_tiles);
    if (t->compact_grid > max_tiles) t->compact_grid = static_cast<int>(max_tiles);

    if (t->stream) {
        t->gstream = t->stream;
    } else {
        if (cudaStreamCreateWithFlags(&t->gstream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(SCLF_ECUDA);
        t->own_gstream = true;
    }
    if (cudaEventCreateWithFlags(&t->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(SCLF_ECUDA);
    *out = t;
    return SCLF_OK;
}

int tube_destroy(tube_t t) {
    if (!t) return SCLF_EINVAL;
    if (t->stream || t->gstream) cudaStreamSynchronize(t->stream);
    if (t->chunk) cudaGraphExecDestroy(t->chunk);
    for (auto& c : t->tchunk) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        for (cudaEvent_t e : c.ev) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : t->ev) cudaEventDestroy(e);
    if (t->fork) cudaEventDestroy(t->fork);
    if (t->join) cudaEventDestroy(t->join);
    if (t->own_gstream && t->gstream) {
        cudaStreamSynchronize(t->gstream);
        cudaStreamDestroy(t->gstream);
    }
    if (t->owns_ws && t->ws) cudaFree(t->ws);
    if (t->sort_ws) cudaFree(t->sort_ws);
    if (t->status_ring) cudaFreeHost(t->status_ring);
    delete t;
    return SCLF_OK;
}

int tube_get_derived(tube_t t, tube_derived* d) {
    if (!t || !d) return SCLF_EINVAL;
    *d = t->d;
    return SCLF_OK;
}

int tube_inject(tube_t t, int64_t* n_injected) {
    if (!t) return SCLF_EINVAL;
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    int64_t n = h.n_inj;
    if (h.n_slots + n > t->p.capacity) return SCLF_ECAPACITY;
    CK(do_append(t, h.n_slots, n, true));
    CK(do_base_weight(t, h.n_slots, n));
    CK(launch_finish_append(t->st, t->ez, n, t->fc, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    if (n_injected) *n_injected = n;
    return SCLF_OK;
}

int tube_add_particles(tube_t t, int64_t n, const double* z, const double* u) {
    if (!t || n < 0 || (n > 0 && (!z || !u))) return SCLF_EINVAL;
    std::vector<char> xs, us;
    const int rc = native_particles(t, n, z, u, xs, us);
    if (rc) return rc;
    return append_raw(t, n, xs.data(), us.data(), nullptr);
}

int tube_step(tube_t t) {
    NvtxRange nvtx_range("tube_step");
    if (!t) return SCLF_EINVAL;
    if (t->owned) return SCLF_ESTATE;
    return one_step(t);
}

int tube_run(tube_t t, int64_t nsteps) {
    NvtxRange nvtx_range("tube_run");
    if (!t || nsteps < 0) return SCLF_EINVAL;
    if (t->owned) return SCLF_ESTATE;
    while (nsteps > 0) {
        if (t->p.sort_interval > 0 && t->steps_since_sort >= t->p.sort_interval) {
            const int rc = tube_sort(t);
            if (rc) return rc;
        }
        if (t->p.use_graphs && (t->host_step & 1) == 0 &&
            t->steps_since_compact == 0 && nsteps >= t->chunk_steps) {
            int rc;
            if (t->timing && (t->timing_tick++ % t->timing_every) == 0) {
                rc = launch_timed_chunk(t);
            } else {
                rc = build_chunk(t);
                if (!rc) rc = launch_chunk(t);
            }
            if (rc) return rc;
            if (t->timing) {
                t->acc.steps_run += t->chunk_steps;
                t->acc.compactions_run += 1;
            }
            nsteps -= t->chunk_steps;
            t->steps_since_sort += t->chunk_steps;
            continue;
        }
        const int rc = one_step(t);
        if (rc) return rc;
        nsteps -= 1;
        t->steps_since_sort += 1;
    }
    return SCLF_OK;
}

int tube_selftest_wait_timeout(tube_t t) {
    if (!t) return SCLF_EINVAL;
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    const int64_t tile = fp64(t) ? Layout<double>::kTile : Layout<float>::kTile;
    if (h.n_slots <= tile) return SCLF_EINVAL;          // needs a second tile to wait
    CK(cudaMemsetAsync(&t->st->ticket, 0, sizeof(unsigned int), t->stream));
    cudaError_t e;
    if (fix32(t)) {
        auto a = compact_args<int, float>(t, 1);
        a.withhold_first = 1;
        a.spin_limit = 4096;
        e = launch_compact<int, float>(a, t->compact_grid, t->stream);
    } else if (fp64(t)) {
        auto a = compact_args<double, double>(t, 1);
        a.withhold_first = 1;
        a.spin_limit = 4096;
        e = launch_compact<double, double>(a, t->compact_grid, t->stream);
    } else {
        auto a = compact_args<float, float>(t, 1);
        a.withhold_first = 1;
        a.spin_limit = 4096;
        e = launch_compact<float, float>(a, t->compact_grid, t->stream);
    }
    CK(e);
    rc = read_state(t, &h);
    if (rc) return rc;
    return (h.flags & SCLF_FLAG_TIMEOUT) ? SCLF_ETIMEOUT : SCLF_OK;
}

int tube_selftest_velocity(uint32_t first, uint64_t count, uint64_t* n_mismatch,
                           uint32_t* first_mismatch) {
    if (!n_mismatch || !first_mismatch) return SCLF_EINVAL;
    if (count > (uint64_t(1) << 32) - first) return SCLF_EINVAL;
    *n_mismatch = 0;
    *first_mismatch = 0xffffffffu;
    if (count == 0) return SCLF_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SCLF_ECUDA;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return SCLF_ENOMEM;
    const unsigned long long init[2] = {0ULL, ~0ULL};
    unsigned long long h[2] = {0ULL, ~0ULL};
    cudaError_t e = cudaMemcpy(d, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_velocity_check(first, count, d, sms * 8, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return SCLF_ECUDA;
    *n_mismatch = h[0];
    *first_mismatch = h[0] ? static_cast<uint32_t>(h[1]) : 0xffffffffu;
    return SCLF_OK;
}

int tube_sort(tube_t t) {
    NvtxRange nvtx_range("tube_sort");
    if (!t) return SCLF_EINVAL;
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    const int64_t n = h.n_slots;
    t->steps_since_sort = 0;
    if (n == 0) return SCLF_OK;
    const int64_t rs = fp64(t) ? 8 : 4;
    const int64_t cap = t->lay.cap_pad;
    const int64_t sb = (sort_scratch_bytes(cap) + 255) / 256 * 256;
    const int64_t gb = (cap * rs + 255) / 256 * 256;
    if (!t->sort_ws) {
        const int64_t bytes = sb + 2 * gb + (t->ids ? cap * 8 : 0);
        if (cudaMalloc(&t->sort_ws, bytes) != cudaSuccess) { t->sort_ws = nullptr; return SCLF_ENOMEM; }
    }
    void* gx = t->sort_ws + sb;
    void* gu = t->sort_ws + sb + gb;
    long long* gi = t->ids ? reinterpret_cast<long long*>(t->sort_ws + sb + 2 * gb) : nullptr;
    const int nz = static_cast<int>(t->p.Nz);
    cudaError_t e;
    if (fp64(t))
        e = launch_sort_by_cell<double, double>(static_cast<const double*>(t->xi),
                                                static_cast<const double*>(t->u), t->ids, n, nz,
                                                1.0, t->sort_ws, static_cast<double*>(gx),
                                                static_cast<double*>(gu), gi, t->stream);
    else if (fix32(t))
        e = launch_sort_by_cell<int, float>(static_cast<const int*>(t->xi),
                                            static_cast<const float*>(t->u), t->ids, n, nz,
                                            std::ldexp(1.0, -t->fb), t->sort_ws,
                                            static_cast<int*>(gx), static_cast<float*>(gu), gi,
                                            t->stream);
    else
        e = launch_sort_by_cell<float, float>(static_cast<const float*>(t->xi),
                                              static_cast<const float*>(t->u), t->ids, n, nz,
                                              1.0, t->sort_ws, static_cast<float*>(gx),
                                              static_cast<float*>(gu), gi, t->stream);
    CK(e);
    // the live particles now fill slots [0, n_live) in cell order; holes drop out
    const int64_t live = h.n_live;
    CK(cudaMemcpyAsync(t->xi, gx, live * rs, cudaMemcpyDeviceToDevice, t->stream));
    CK(cudaMemcpyAsync(t->u, gu, live * rs, cudaMemcpyDeviceToDevice, t->stream));
    if (gi) CK(cudaMemcpyAsync(t->ids, gi, live * 8, cudaMemcpyDeviceToDevice, t->stream));
    CK(cudaMemcpyAsync(&t->st->n_slots, &live, sizeof(long long), cudaMemcpyHostToDevice,
                       t->stream));
    CK(cudaStreamSynchronize(t->stream));
    t->steps_since_compact = 0;
    return SCLF_OK;
}

int tube_read_fields(tube_t t, double* Ez, double* Er, double* Bphi, double* J, double* rho) {
    if (!t) return SCLF_EINVAL;
    const int64_t nz = t->p.Nz;
    const int par = static_cast<int>(t->host_step & 1);
    CK(cudaStreamSynchronize(t->stream));
    if (Ez) CK(cudaMemcpyAsync(Ez, t->ez, nz * 8, cudaMemcpyDeviceToHost, t->stream));
    if (Er) CK(cudaMemcpyAsync(Er, t->er[par], (nz + 1) * 8, cudaMemcpyDeviceToHost, t->stream));
    if (Bphi) CK(cudaMemcpyAsync(Bphi, t->b[par], nz * 8, cudaMemcpyDeviceToHost, t->stream));
    if (J) CK(cudaMemcpyAsync(J, t->jlast, nz * 8, cudaMemcpyDeviceToHost, t->stream));
    if (rho) {
        DevState h;
        int rc = read_state(t, &h);
        if (rc) return rc;
        CK(cudaMemsetAsync(t->rho_acc, 0, (nz + 1) * 8, t->stream));
        CK(do_rho(t, h.n_slots));
        CK(cudaMemcpyAsync(rho, t->rho_acc, (nz + 1) * 8, cudaMemcpyDeviceToHost, t->stream));
    }
    CK(cudaStreamSynchronize(t->stream));
    if (rho) {
        const double scale = t->d.s / t->d.dz;     // rho_j = s * sum(w) / dz
        for (int64_t j = 0; j <= nz; ++j) rho[j] *= scale;
    }
    return SCLF_OK;
}

// Live particles in ID order: a forced (stable) compaction on the device
// first, so that slots [0, n_live) hold them without holes; then one copy per
// array straight into the caller's memory (convert: z = xi dz and u as
// double, through host staging).
static int read_raw(tube_t t, int64_t cap, int64_t* n, void* xo, void* uo, int64_t* ido,
                    bool convert) {
    NvtxRange nvtx_range("tube_read_particles");
    CK(enqueue_compact(t, t->stream, 1));
    t->steps_since_compact = 0;
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    if (h.flags & SCLF_FLAG_TIMEOUT) return SCLF_ETIMEOUT;
    const int64_t ns = h.n_slots;                    // == live particles after compaction
    const int64_t m = ns < cap ? ns : cap;
    const int64_t rs = fp64(t) ? 8 : 4;
    if (m > 0) {
        if (convert) {
            std::vector<char> xs(m * rs), us(m * rs);
            CK(cudaMemcpyAsync(xs.data(), t->xi, m * rs, cudaMemcpyDeviceToHost, t->stream));
            CK(cudaMemcpyAsync(us.data(), t->u, m * rs, cudaMemcpyDeviceToHost, t->stream));
            if (ido && t->ids)
                CK(cudaMemcpyAsync(ido, t->ids, m * 8, cudaMemcpyDeviceToHost, t->stream));
            CK(cudaStreamSynchronize(t->stream));
            for (int64_t i = 0; i < m; ++i) {
                if (xo) static_cast<double*>(xo)[i] = raw_cells(t, xs.data(), i) * t->d.dz;
                if (uo) static_cast<double*>(uo)[i] = raw_mom(t, us.data(), i);
            }
        } else {
            if (xo) CK(cudaMemcpyAsync(xo, t->xi, m * rs, cudaMemcpyDeviceToHost, t->stream));
            if (uo) CK(cudaMemcpyAsync(uo, t->u, m * rs, cudaMemcpyDeviceToHost, t->stream));
            if (ido && t->ids)
                CK(cudaMemcpyAsync(ido, t->ids, m * 8, cudaMemcpyDeviceToHost, t->stream));
            CK(cudaStreamSynchronize(t->stream));
        }
        if (ido && !t->ids)
            for (int64_t i = 0; i < m; ++i) ido[i] = -1;
    }
    if (n) *n = ns;
    return SCLF_OK;
}

int tube_read_particles(tube_t t, int64_t cap, int64_t* n, double* z, double* u, int64_t* id) {
    if (!t || cap < 0) return SCLF_EINVAL;
    return read_raw(t, cap, n, z, u, id, true);
}

int tube_save_particles(tube_t t, int64_t cap, int64_t* n, void* xi, void* u, int64_t* id) {
    if (!t || cap < 0) return SCLF_EINVAL;
    return read_raw(t, cap, n, xi, u, id, false);
}

int tube_load_particles(tube_t t, int64_t n, const void* xi, const void* u, const int64_t* id) {
    NvtxRange nvtx_range("tube_load_particles");
    if (!t || n < 0 || n > t->p.capacity || (n > 0 && (!xi || !u))) return SCLF_EINVAL;
    if (id && !t->ids) return SCLF_EINVAL;
    // the counters start from an empty tube; the raw arrays go straight to
    // the slots and are checked on the device
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    h.n_slots = 0;
    h.n_live = 0;
    h.total_injected = 0;
    h.w0 = 0;
    h.acc_w0 = 0;
    h.load_bad = 0;
    h.max_id = -1;
    CK(cudaMemcpyAsync(t->st, &h, sizeof(h), cudaMemcpyHostToDevice, t->stream));
    const int64_t rs = fp64(t) ? 8 : 4;
    if (n > 0) {
        CK(cudaMemcpyAsync(t->xi, xi, n * rs, cudaMemcpyHostToDevice, t->stream));
        CK(cudaMemcpyAsync(t->u, u, n * rs, cudaMemcpyHostToDevice, t->stream));
        if (id) CK(cudaMemcpyAsync(t->ids, id, n * 8, cudaMemcpyHostToDevice, t->stream));
        else if (t->ids) CK(do_append(t, 0, n, false));       // IDs 0..n-1
        const long long* dev_ids = id ? t->ids : nullptr;
        if (fp64(t)) {
            CK((launch_validate<double, double>(t->st, static_cast<const double*>(t->xi),
                                                static_cast<const double*>(t->u), dev_ids, n,
                                                double(t->p.Nz), t->stream)));
        } else if (fix32(t)) {
            CK((launch_validate<int, float>(t->st, static_cast<const int*>(t->xi),
                                            static_cast<const float*>(t->u), dev_ids, n,
                                            std::ldexp(double(t->p.Nz), t->fb), t->stream)));
        } else {
            CK((launch_validate<float, float>(t->st, static_cast<const float*>(t->xi),
                                              static_cast<const float*>(t->u), dev_ids, n,
                                              double(t->p.Nz), t->stream)));
        }
        CK(do_base_weight(t, 0, n));
    }
    CK(launch_finish_append(t->st, t->ez, n, t->fc, t->stream));
    rc = read_state(t, &h);
    if (rc) return rc;
    if (h.load_bad) {
        // leave an empty tube rather than particles that failed the check
        h.n_slots = h.n_live = h.total_injected = h.w0 = 0;
        h.load_bad = 0;
        CK(cudaMemcpyAsync(t->st, &h, sizeof(h), cudaMemcpyHostToDevice, t->stream));
        CK(launch_finish_append(t->st, t->ez, 0, t->fc, t->stream));
        CK(cudaStreamSynchronize(t->stream));
        return SCLF_EINVAL;
    }
    if (id && h.max_id + 1 > h.total_injected) {   // IDs continue after the largest loaded one
        h.total_injected = h.max_id + 1;
        CK(cudaMemcpyAsync(&t->st->total_injected, &h.total_injected, sizeof(long long),
                           cudaMemcpyHostToDevice, t->stream));
        CK(cudaStreamSynchronize(t->stream));
    }
    return SCLF_OK;
}

int tube_solve_fields(tube_t t) {
    NvtxRange nvtx_range("tube_solve_fields");
    if (!t) return SCLF_EINVAL;
    const int64_t nz = t->p.Nz;
    std::vector<double> rho(nz + 1), src(nz + 1), phi(nz + 1), ez0(nz);
    int rc = tube_read_fields(t, nullptr, nullptr, nullptr, nullptr, rho.data());
    if (rc) return rc;
    // phi'' - phi = 4 pi (rho_GJ - rho)
    for (int64_t j = 0; j <= nz; ++j) src[j] = t->rho_gj[j] - rho[j];
    solve_poisson(src.data(), nz, t->d.dz, phi.data());
    for (int64_t j = 0; j < nz; ++j) ez0[j] = -(phi[j + 1] - phi[j]) / t->d.dz;
    return set_fields_host(t, ez0.data(), phi.data(), nullptr);   // E_r = phi / R, B = 0
}

int tube_diagnostics(tube_t t, tube_diag* out) {
    if (!t || !out) return SCLF_EINVAL;
    NvtxRange nvtx_range("tube_diagnostics");
    DevState h;
    int rc = read_state(t, &h);
    if (rc) return rc;
    double pd[3] = {0.0, 0.0, 0.0};
    if (h.n_slots > 0) {
        cudaError_t e;
        double* part = t->diag;
        double* res = t->diag + 3 * kDiagBlocks;
        if (fp64(t))
            e = launch_particle_diag<double, double>(static_cast<const double*>(t->xi),
                                                     static_cast<const double*>(t->u), h.n_slots,
                                                     part, res, t->stream);
        else if (fix32(t))
            e = launch_particle_diag<int, float>(static_cast<const int*>(t->xi),
                                                 static_cast<const float*>(t->u), h.n_slots, part,
                                                 res, t->stream);
        else
            e = launch_particle_diag<float, float>(static_cast<const float*>(t->xi),
                                                   static_cast<const float*>(t->u), h.n_slots,
                                                   part, res, t->stream);
        CK(e);
        CK(cudaMemcpyAsync(pd, res, sizeof(pd), cudaMemcpyDeviceToHost, t->stream));
    }
    const int64_t nz = t->p.Nz;
    std::vector<double> ez(nz), er(nz + 1), b(nz), rho(nz + 1);
    rc = tube_read_fields(t, ez.data(), er.data(), b.data(), nullptr, rho.data());
    if (rc) return rc;
    const double dz = t->d.dz;
    double fe = 0.0;
    for (int64_t j = 0; j < nz; ++j) fe += (ez[j] * ez[j] + b[j] * b[j]) * dz;
    for (int64_t j = 0; j <= nz; ++j) fe += er[j] * er[j] * dz * ((j == 0 || j == nz) ? 0.5 : 1.0);
    double gmax = 0.0, gscale = 0.0;
    for (int64_t j = 1; j < nz; ++j) {
        const double src = 4.0 * kPi * (rho[j] - t->rho_gj[j]);
        const double g = (ez[j] - ez[j - 1]) / dz + er[j] - src;
        gmax = std::fmax(gmax, std::fabs(g));
        gscale = std::fmax(gscale, std::fabs(src));
    }
    out->n_particles = static_cast<int64_t>(pd[0]);
    out->gamma_max = pd[2];
    out->gamma_mean = pd[0] > 0.0 ? pd[1] / pd[0] : 0.0;
    out->kinetic = (pd[1] - pd[0]) * std::fabs(t->d.s);
    out->field_energy = fe / (8.0 * kPi);
    out->gauss_max = gmax;
    out->gauss_scale = gscale;
    return SCLF_OK;
}

int tube_status(tube_t t, tube_stats* out) {
    if (!t || !out) return SCLF_EINVAL;
    DevState h;
    const int rc = read_state(t, &h);
    if (rc) return rc;
    stats_from_state(h, out);
    return SCLF_OK;
}

int tube_status_async(tube_t t, int64_t* ticket) {
    if (!t || !ticket) return SCLF_EINVAL;
    if (!t->status_ring) {
        void* p = nullptr;
        if (cudaHostAlloc(&p, sizeof(DevState) * sclf_tube::kStatusRing, cudaHostAllocDefault) !=
            cudaSuccess)
            return SCLF_ENOMEM;
        t->status_ring = static_cast<DevState*>(p);
    }
    const int64_t k = t->status_next;
    CK(cudaMemcpyAsync(t->status_ring + k % sclf_tube::kStatusRing, t->st, sizeof(DevState),
                       cudaMemcpyDeviceToHost, t->stream));
    t->status_next = k + 1;
    *ticket = k;
    return SCLF_OK;
}

int tube_status_collect(tube_t t, int64_t ticket, tube_stats* out) {
    if (!t || !out || !t->status_ring || ticket < 0 || ticket >= t->status_next ||
        ticket < t->status_next - sclf_tube::kStatusRing)
        return SCLF_EINVAL;
    CK(cudaStreamSynchronize(t->stream));
    stats_from_state(t->status_ring[ticket % sclf_tube::kStatusRing], out);
    return SCLF_OK;
}

int tube_check(tube_t t) {
    tube_stats s;
    const int rc = tube_status(t, &s);
    if (rc) return rc;
    if (s.flags & SCLF_FLAG_BOUNDS) return SCLF_EBOUNDS;
    if (s.flags & SCLF_FLAG_TIMEOUT) return SCLF_ETIMEOUT;
    if (s.flags & SCLF_FLAG_NONFINITE) return SCLF_ENONFINITE;
    if (s.flags & SCLF_FLAG_CAPACITY) return SCLF_ECAPACITY;
    return SCLF_OK;
}

int tube_compact(tube_t t) {
    if (!t) return SCLF_EINVAL;
    CK(enqueue_compact(t, t->stream, 1));
    t->steps_since_compact = 0;
    return SCLF_OK;
}

int tube_set_timing(tube_t t, int enable) {
    if (!t || enable < 0) return SCLF_EINVAL;
    if (enable) {
        if (t->ev.empty()) {
            t->ev.resize(3 * 2048 + 8, nullptr);
            for (auto& e : t->ev)
                if (cudaEventCreate(&e) != cudaSuccess) return SCLF_ECUDA;
        }
        CK(cudaStreamSynchronize(t->stream));
        t->recs.clear();
        t->ev_next = 0;
        for (auto& c : t->tchunk) c.pending = false;   // discard an earlier session
        std::memset(&t->acc, 0, sizeof(t->acc));
        DevState h;
        const int rc = read_state(t, &h);
        if (rc) return rc;
        t->slots_base = h.slots_processed;
        t->timing = true;
        t->timing_every = enable;
        t->timing_tick = 0;
    } else {
        const int rc = drain_timing(t);
        t->timing = false;
        return rc;
    }
    return SCLF_OK;
}

int tube_get_timing(tube_t t, tube_timing* out) {
    if (!t || !out) return SCLF_EINVAL;
    int rc = drain_timing(t);
    if (rc) return rc;
    DevState h;
    rc = read_state(t, &h);
    if (rc) return rc;
    *out = t->acc;
    out->particle_slots = static_cast<int64_t>(h.slots_processed - t->slots_base);
    return SCLF_OK;
}

const char* tube_strerror(int code) {
    switch (code) {
        case SCLF_OK: return "ok";
        case SCLF_EINVAL: return "invalid argument";
        case SCLF_ENOMEM: return "out of memory or workspace too small";
        case SCLF_ECUDA: return "CUDA runtime error";
        case SCLF_ECAPACITY: return "particle capacity exhausted";
        case SCLF_ENONFINITE: return "non-finite particle state";
        case SCLF_ETIMEOUT: return "device-side wait timed out";
        case SCLF_ESTATE: return "invalid state for this call";
        case SCLF_EBOUNDS: return "index out of bounds (bounds-checked build)";
        default: return "unknown error";
    }
}

const char* tube_version(void) {
#ifdef SCLF_CHECKED
    return "sclf_tube 0.1.0 sm_103a bounds-checked";
#else
    return "sclf_tube 0.1.0 sm_103a";
#endif
}

}  // extern "C"

// ===========================================================================
// Batches: many independent tubes advanced by one particle launch and one
// field launch per step.
// ===========================================================================
struct sclf_batch {
    std::vector<sclf_tube*> tubes;
    cudaStream_t stream = nullptr;
    cudaStream_t gstream = nullptr;
    bool own_gstream = false;
    cudaEvent_t fork = nullptr, join = nullptr;
    // one descriptor array and tile-to-tube table per tile size of the
    // particle kernel's shapes (tile0 differs between them)
    BatchTube* d_desc[3] = {nullptr, nullptr, nullptr};
    int* d_tile_tube[3] = {nullptr, nullptr, nullptr};
    int* d_cell_tube = nullptr;
    tube_stats* d_stats = nullptr;     // batch_status gathers every tube's counters here
    long long n_tiles[3] = {0, 0, 0};
    int n_cells = 0;
    int push_grid[kBatchVariants] = {};
    // the tubes' constants by value for the particle kernel (batches of up to
    // kBatchConstTubes tubes), one table per tile class (tile0 differs)
    std::vector<BatchConstTable> ctab;
    int const_grid[kBatchVariants] = {};
    int variant = 0;                   // particle kernel shape (batch_autotune)
    bool fix32 = false;                // SCLF_FIX32 tubes: one particle-kernel shape
    int fix_grid = 0;
    bool overlap = true;               // step kernels by programmatic dependent launch
    int64_t host_step = 0;
    int steps_since_compact = 0;
    int compact_every = 64;
    int chunk_steps = 64;
    cudaGraphExec_t chunk = nullptr;
    bool timing = false;
    int timing_every = 1;              // sampling period (steps)
    int64_t timing_tick = 0;
    std::vector<cudaEvent_t> ev;       // 3 per step, 2 per compaction round
    std::vector<std::pair<int, int>> recs;
    int ev_next = 0;
    tube_timing acc{};
    std::vector<unsigned long long> slots_base;
};

namespace {

// Tile-size class of a particle-kernel shape: 0 for kThreads * 8 slots, 1
// for kThreads * 4, 2 for kThreads * 16.
constexpr int kTileClasses = 3;
constexpr int kClassPPT[kTileClasses] = {8, 4, 16};
int tile_class(int variant) {
    const int ppt = kBatchPPT[variant];
    return ppt == 8 ? 0 : (ppt == 4 ? 1 : 2);
}

cudaError_t batch_launch_push(sclf_batch* b, cudaStream_t s) {
    if (b->fix32) {
        const cudaError_t e = launch_batch_refresh(b->d_desc[0], static_cast<int>(b->tubes.size()),
                                                   s, b->overlap);
        if (e != cudaSuccess) return e;
        return launch_batch_push_fix32(b->d_desc[0], b->d_tile_tube[0], b->n_tiles[0], b->fix_grid,
                                       s, b->overlap);
    }
    const int c = tile_class(b->variant);
    const cudaError_t e = launch_batch_refresh(b->d_desc[c], static_cast<int>(b->tubes.size()), s,
                                               b->overlap);
    if (e != cudaSuccess) return e;
    if (!b->ctab.empty())
        return launch_batch_push_const(b->ctab[c], b->d_desc[c], b->d_tile_tube[c], b->n_tiles[c],
                                       b->const_grid[b->variant], b->variant, s, b->overlap);
    return launch_batch_push(b->d_desc[c], b->d_tile_tube[c], b->n_tiles[c],
                             b->push_grid[b->variant], b->variant, s, b->overlap);
}

int batch_enqueue_step(sclf_batch* b, cudaStream_t s, int parity) {
    CK(batch_launch_push(b, s));
    CK(launch_batch_field(b->d_desc[0], b->d_cell_tube, b->n_cells, parity, s, b->overlap));
    return SCLF_OK;
}

int batch_enqueue_compaction(sclf_batch* b, cudaStream_t s) {
    for (sclf_tube* t : b->tubes) CK(enqueue_compact(t, s, 0));
    return SCLF_OK;
}

void batch_advance(sclf_batch* b, int64_t n) {
    b->host_step += n;
    for (sclf_tube* t : b->tubes) t->host_step += n;
}

int batch_drain(sclf_batch* b) {
    CK(cudaStreamSynchronize(b->stream));
    for (const auto& r : b->recs) {
        float ms = 0.f;
        if (r.first == 0) {
            CK(cudaEventElapsedTime(&ms, b->ev[r.second], b->ev[r.second + 1]));
            b->acc.push_ms += ms;
            CK(cudaEventElapsedTime(&ms, b->ev[r.second + 1], b->ev[r.second + 2]));
            b->acc.field_ms += ms;
            b->acc.n_steps += 1;
        } else {
            CK(cudaEventElapsedTime(&ms, b->ev[r.second], b->ev[r.second + 1]));
            b->acc.compact_ms += ms;
            b->acc.n_compactions += 1;
        }
    }
    b->recs.clear();
    b->ev_next = 0;
    return SCLF_OK;
}

int batch_reserve(sclf_batch* b, int k) {
    if (b->ev_next + k > static_cast<int>(b->ev.size()))
        if (batch_drain(b) != SCLF_OK) return -1;
    if (b->ev_next + k > static_cast<int>(b->ev.size())) return -1;
    const int e0 = b->ev_next;
    b->ev_next += k;
    return e0;
}

int batch_one_step(sclf_batch* b) {
    const int parity = static_cast<int>(b->host_step & 1);
    const bool timed = b->timing && (b->timing_tick++ % b->timing_every) == 0;
    if (timed) {
        const int e0 = batch_reserve(b, 3);
        if (e0 < 0) return SCLF_ECUDA;
        CK(cudaEventRecord(b->ev[e0], b->stream));
        CK(batch_launch_push(b, b->stream));
        CK(cudaEventRecord(b->ev[e0 + 1], b->stream));
        CK(launch_batch_field(b->d_desc[0], b->d_cell_tube, b->n_cells, parity, b->stream,
                              b->overlap));
        CK(cudaEventRecord(b->ev[e0 + 2], b->stream));
        b->recs.push_back({0, e0});
    } else {
        const int rc = batch_enqueue_step(b, b->stream, parity);
        if (rc) return rc;
    }
    batch_advance(b, 1);
    if (b->timing) b->acc.steps_run += 1;
    if (++b->steps_since_compact >= b->compact_every) {
        if (b->timing) b->acc.compactions_run += 1;
        int e0 = -1;
        if (b->timing) {
            e0 = batch_reserve(b, 2);
            if (e0 < 0) return SCLF_ECUDA;
            CK(cudaEventRecord(b->ev[e0], b->stream));
        }
        const int rc = batch_enqueue_compaction(b, b->stream);
        if (rc) return rc;
        if (b->timing) {
            CK(cudaEventRecord(b->ev[e0 + 1], b->stream));
            b->recs.push_back({1, e0});
        }
        b->steps_since_compact = 0;
    }
    return SCLF_OK;
}

int batch_build_chunk(sclf_batch* b) {
    if (b->chunk) return SCLF_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = SCLF_OK;
    for (int k = 0; k < b->chunk_steps && rc == SCLF_OK; ++k) rc = batch_enqueue_step(b, b->gstream, k & 1);
    if (rc == SCLF_OK) rc = batch_enqueue_compaction(b, b->gstream);
    const cudaError_t e2 = cudaStreamEndCapture(b->gstream, &g);
    if (rc != SCLF_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e2);
    const cudaError_t e = cudaGraphInstantiate(&b->chunk, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return SCLF_OK;
}

}  // namespace

extern "C" {

int batch_create(int32_t n, const tube_params* params, void* stream, batch_t* out) {
    if (!out || n <= 0 || !params) return SCLF_EINVAL;
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i)
        if ((params[i].precision != SCLF_FP32 && params[i].precision != SCLF_FIX32) ||
            params[i].precision != params[0].precision ||
            params[i].accumulate != SCLF_ACC_FIXED64)
            return SCLF_EINVAL;
    sclf_batch* b = new (std::nothrow) sclf_batch();
    if (!b) return SCLF_ENOMEM;
    b->stream = static_cast<cudaStream_t>(stream);
    b->fix32 = params[0].precision == SCLF_FIX32;
    b->overlap = params[0].launch_overlap >= 0;
    auto fail = [&](int code) { batch_destroy(b); return code; };
    std::vector<BatchTube> desc(n);
    std::vector<int> tile_tube[kTileClasses], cell_tube;
    long long tiles[kTileClasses] = {0, 0, 0};
    long long cells = 0;
    b->compact_every = params[0].compact_interval > 0 ? params[0].compact_interval : 64;
    b->chunk_steps = b->compact_every + (b->compact_every & 1);
    std::vector<long long> tile0[kTileClasses];
    for (int32_t i = 0; i < n; ++i) {
        tube_t t = nullptr;
        const int rc = tube_create(&params[i], nullptr, 0, stream, &t);
        if (rc) return fail(rc);
        t->owned = true;
        b->tubes.push_back(t);
        BatchTube& d = desc[i];
        d.st = t->st;
        d.xi = static_cast<float*>(t->xi);
        d.u = static_cast<float*>(t->u);
        d.ids = t->ids;
        d.ez2 = static_cast<float*>(t->ez2);
        d.jacc = static_cast<long long*>(t->jacc);
        d.capacity = t->p.capacity;
        d.tile0 = 0;
        d.n_slots = d.n_tot = d.id0 = d.n_req = 0;
        d.nz = static_cast<int>(t->p.Nz);
        d.cell0 = static_cast<int>(cells);
        d.nzf = static_cast<float>(t->p.Nz);
        d.dt = static_cast<float>(t->d.dt);
        d.cfl = static_cast<float>(t->d.dt / t->d.dz);
        d.ez = t->ez;
        d.er[0] = t->er[0];
        d.er[1] = t->er[1];
        d.b[0] = t->b[0];
        d.b[1] = t->b[1];
        d.jlast = t->jlast;
        d.fc = t->fc;
        d.fb = t->fb;
        for (int c = 0; c < kTileClasses; ++c) {   // cap_pad is a multiple of every tile size
            const long long nt = t->lay.cap_pad / (kThreads * static_cast<long long>(kClassPPT[c]));
            tile0[c].push_back(tiles[c]);
            tile_tube[c].insert(tile_tube[c].end(), static_cast<size_t>(nt), i);
            tiles[c] += nt;
        }
        cell_tube.insert(cell_tube.end(), static_cast<size_t>(t->p.Nz), i);
        cells += t->p.Nz;
        if (cells >= (1LL << 31)) return fail(SCLF_EINVAL);
    }
    b->n_cells = static_cast<int>(cells);
    if (n <= kBatchConstTubes && !b->fix32) {
        try {
            b->ctab.resize(kTileClasses);
        } catch (...) {
            return fail(SCLF_ENOMEM);
        }
        for (int c = 0; c < kTileClasses; ++c) {
            BatchConstTable& k = b->ctab[c];
            std::memset(&k, 0, sizeof(k));
            for (int32_t i = 0; i < n; ++i) {
                const BatchTube& d = desc[i];
                k.t[i] = BatchConst{d.st, d.xi, d.u, d.ids, d.ez2, d.jacc, tile0[c][i], d.nz, d.nzf,
                                    d.dt, d.cfl};
            }
        }
    }
    for (int c = 0; c < kTileClasses; ++c) {
        std::vector<BatchTube> dc(desc);
        for (int32_t i = 0; i < n; ++i) dc[i].tile0 = tile0[c][i];
        b->n_tiles[c] = tiles[c];
        if (cudaMalloc(&b->d_desc[c], sizeof(BatchTube) * n) != cudaSuccess ||
            cudaMalloc(&b->d_tile_tube[c], sizeof(int) * tiles[c]) != cudaSuccess)
            return fail(SCLF_ENOMEM);
        if (cudaMemcpyAsync(b->d_desc[c], dc.data(), sizeof(BatchTube) * n, cudaMemcpyHostToDevice,
                            b->stream) ||
            cudaMemcpyAsync(b->d_tile_tube[c], tile_tube[c].data(), sizeof(int) * tiles[c],
                            cudaMemcpyHostToDevice, b->stream) ||
            cudaStreamSynchronize(b->stream))
            return fail(SCLF_ECUDA);
    }
    if (cudaMalloc(&b->d_cell_tube, sizeof(int) * cells) != cudaSuccess) return fail(SCLF_ENOMEM);
    if (cudaMalloc(&b->d_stats, sizeof(tube_stats) * n) != cudaSuccess) return fail(SCLF_ENOMEM);
    if (cudaMemcpyAsync(b->d_cell_tube, cell_tube.data(), sizeof(int) * cells, cudaMemcpyHostToDevice, b->stream) ||
        cudaStreamSynchronize(b->stream))
        return fail(SCLF_ECUDA);
    const int sms = b->tubes[0]->sms;
    for (int v = 0; v < kBatchVariants; ++v) {
        b->push_grid[v] = batch_push_grid_size(v, sms);
        b->const_grid[v] = batch_push_const_grid_size(v, sms);
        const long long nt = b->n_tiles[tile_class(v)];
        if (b->push_grid[v] > nt) b->push_grid[v] = static_cast<int>(nt);
        if (b->const_grid[v] > nt) b->const_grid[v] = static_cast<int>(nt);
    }
    b->fix_grid = batch_push_fix32_grid_size(sms);
    if (b->fix_grid > b->n_tiles[0]) b->fix_grid = static_cast<int>(b->n_tiles[0]);
    if (b->stream) {
        b->gstream = b->stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(SCLF_ECUDA);
        b->own_gstream = true;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(SCLF_ECUDA);
    *out = b;
    return SCLF_OK;
}

int batch_destroy(batch_t b) {
    if (!b) return SCLF_EINVAL;
    cudaStreamSynchronize(b->stream);
    if (b->chunk) cudaGraphExecDestroy(b->chunk);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->own_gstream && b->gstream) {
        cudaStreamSynchronize(b->gstream);
        cudaStreamDestroy(b->gstream);
    }
    for (sclf_tube* t : b->tubes) tube_destroy(t);
    for (int c = 0; c < kTileClasses; ++c) {
        if (b->d_desc[c]) cudaFree(b->d_desc[c]);
        if (b->d_tile_tube[c]) cudaFree(b->d_tile_tube[c]);
    }
    if (b->d_cell_tube) cudaFree(b->d_cell_tube);
    if (b->d_stats) cudaFree(b->d_stats);
    delete b;
    return SCLF_OK;
}

int batch_size(batch_t b, int32_t* n) {
    if (!b || !n) return SCLF_EINVAL;
    *n = static_cast<int32_t>(b->tubes.size());
    return SCLF_OK;
}

int batch_tube(batch_t b, int32_t i, tube_t* out) {
    if (!b || !out || i < 0 || i >= static_cast<int32_t>(b->tubes.size())) return SCLF_EINVAL;
    *out = b->tubes[i];
    return SCLF_OK;
}

int batch_status(batch_t b, int32_t n, tube_stats* out) {
    if (!b || !out || n != static_cast<int32_t>(b->tubes.size())) return SCLF_EINVAL;
    CK(launch_batch_status(b->d_desc[0], n, b->d_stats, b->stream));
    CK(cudaMemcpyAsync(out, b->d_stats, sizeof(tube_stats) * n, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return SCLF_OK;
}

int batch_step(batch_t b) {
    NvtxRange nvtx_range("batch_step");
    if (!b) return SCLF_EINVAL;
    return batch_one_step(b);
}

int batch_run(batch_t b, int64_t nsteps) {
    NvtxRange nvtx_range("batch_run");
    if (!b || nsteps < 0) return SCLF_EINVAL;
    while (nsteps > 0) {
        // timed steps are launched on their own; with a sampling period the
        // others may replay the graph
        const bool graph_ok = !b->timing || b->timing_every > 1;
        if (graph_ok && (b->host_step & 1) == 0 && b->steps_since_compact == 0 &&
            nsteps >= b->chunk_steps && b->tubes[0]->p.use_graphs) {
            int rc = batch_build_chunk(b);
            if (rc) return rc;
            if (b->gstream != b->stream) {
                CK(cudaEventRecord(b->fork, b->stream));
                CK(cudaStreamWaitEvent(b->gstream, b->fork, 0));
            }
            CK(cudaGraphLaunch(b->chunk, b->gstream));
            if (b->gstream != b->stream) {
                CK(cudaEventRecord(b->join, b->gstream));
                CK(cudaStreamWaitEvent(b->stream, b->join, 0));
            }
            batch_advance(b, b->chunk_steps);
            if (b->timing) {
                b->acc.steps_run += b->chunk_steps;
                b->acc.compactions_run += 1;
                b->timing_tick += b->chunk_steps;
            }
            nsteps -= b->chunk_steps;
            continue;
        }
        const int rc = batch_one_step(b);
        if (rc) return rc;
        nsteps -= 1;
    }
    return SCLF_OK;
}

int batch_set_timing(batch_t b, int enable) {
    if (!b || enable < 0) return SCLF_EINVAL;
    if (enable) {
        if (b->ev.empty()) {
            b->ev.resize(3 * 2048 + 8, nullptr);
            for (auto& e : b->ev)
                if (cudaEventCreate(&e) != cudaSuccess) return SCLF_ECUDA;
        }
        CK(cudaStreamSynchronize(b->stream));
        b->recs.clear();
        b->ev_next = 0;
        std::memset(&b->acc, 0, sizeof(b->acc));
        b->slots_base.clear();
        for (sclf_tube* t : b->tubes) {
            DevState h;
            const int rc = read_state(t, &h);
            if (rc) return rc;
            b->slots_base.push_back(h.slots_processed);
        }
        b->timing = true;
        b->timing_every = enable;
        b->timing_tick = 0;
        return SCLF_OK;
    }
    const int rc = batch_drain(b);
    b->timing = false;
    return rc;
}

int batch_set_variant(batch_t b, int32_t variant) {
    if (!b || variant < 0 || variant >= kBatchVariants) return SCLF_EINVAL;
    if (b->fix32 && variant != 0) return SCLF_EINVAL;        // one shape
    if (variant != b->variant && b->chunk) {
        CK(cudaStreamSynchronize(b->stream));
        cudaGraphExecDestroy(b->chunk);          // captured with the previous shape
        b->chunk = nullptr;
    }
    b->variant = variant;
    return SCLF_OK;
}

int batch_autotune(batch_t b, int32_t steps, double* ms, int32_t* chosen) {
    NvtxRange nvtx_range("batch_autotune");
    if (!b || steps <= 0) return SCLF_EINVAL;
    double best = 0.0;
    int best_v = -1;
    if (ms && b->fix32)
        for (int v = 1; v < kBatchVariants; ++v) ms[v] = -1.0;   // shapes not built for FIX32
    for (int v = 0; v < (b->fix32 ? 1 : kBatchVariants); ++v) {
        int rc = batch_set_variant(b, v);
        if (rc) return rc;
        for (int k = 0; k < 2; ++k)              // first launches of this kernel
            if ((rc = batch_one_step(b))) return rc;
        if ((rc = batch_set_timing(b, 1))) return rc;
        for (int k = 0; k < steps; ++k)
            if ((rc = batch_one_step(b))) return rc;
        tube_timing tm;
        if ((rc = batch_get_timing(b, &tm))) return rc;
        if ((rc = batch_set_timing(b, 0))) return rc;
        const double per = tm.push_ms / double(tm.n_steps > 0 ? tm.n_steps : 1);
        if (ms) ms[v] = per;
        if (best_v < 0 || per < best) { best = per; best_v = v; }
    }
    if (chosen) *chosen = best_v;
    return batch_set_variant(b, best_v);
}

int batch_get_timing(batch_t b, tube_timing* out) {
    if (!b || !out) return SCLF_EINVAL;
    int rc = batch_drain(b);
    if (rc) return rc;
    *out = b->acc;
    int64_t slots = 0;
    for (size_t i = 0; i < b->tubes.size(); ++i) {
        DevState h;
        rc = read_state(b->tubes[i], &h);
        if (rc) return rc;
        slots += static_cast<int64_t>(h.slots_processed - (i < b->slots_base.size() ? b->slots_base[i] : 0));
    }
    out->particle_slots = slots;
    return SCLF_OK;
}

}  // extern "C"
