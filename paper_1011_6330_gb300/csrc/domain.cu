// One tube split into contiguous z-ranges of cells (sub-domains), stepped as
// a multi-GPU run would step it, here on one GPU: each sub-domain is a tube
// restricted to its cells (its particle kernel hands particles that leave the
// range to an outbox, its field kernel updates only its cells), and after
// each kernel phase small exchange kernels move what neighbours need (Sec. 2:
// Eq. 3 is local in z and a particle moves less than a cell per step):
//   after the particle kernels: the current deposited across each boundary;
//   after the field kernels: the particles that crossed, then each
//   neighbour's new B_phi and E_z of the boundary cells (the B_phi halo of
//   the next field update and the E_z entries of the next gather table).
// E_r at a shared node is computed by both sides from identical inputs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device_common.cuh"
#include "tube_impl.h"

namespace sclf {
namespace {

constexpr int kMaxDomains = 64;

// What the exchange kernels see of one sub-domain.
struct DomDev {
    DevState* st;
    void* xi;
    void* u;
    long long* ids;
    long long* jacc;
    double* ez;
    double* b[2];
    void* ez2;
    long long capacity;
    int lo, hi;
    Outbox down, up;
};

// Current deposited across boundary c = d[i].hi: sub-domain i's share of cell
// c (owned by i + 1) and i + 1's share of cell c - 1 (owned by i) move to the
// owner; one thread per boundary. Exact integer sums.
__global__ void dom_current_kernel(const DomDev* d, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int c = d[i].hi;
    long long* ja = d[i].jacc;
    long long* jb = d[i + 1].jacc;
    jb[c] += ja[c];
    ja[c] = 0;
    ja[c - 1] += jb[c - 1];
    jb[c - 1] = 0;
}

// Halos after the field update at boundary c = d[i].hi: B_phi^{n+3/2} of the
// cells either side (the next field update reads them) and the gather-table
// components that hold E_z^{n+1} of the neighbour's cell.
template <class Real>
__global__ void dom_halo_kernel(const DomDev* d, int n, int po) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int c = d[i].hi;
    const DomDev& a = d[i];
    const DomDev& b = d[i + 1];
    a.b[po][c] = b.b[po][c];
    b.b[po][c - 1] = a.b[po][c - 1];
    static_cast<Real*>(a.ez2)[2 * c + 1] = static_cast<Real>(b.ez[c]);
    static_cast<Real*>(b.ez2)[2 * c] = static_cast<Real>(a.ez[c - 1]);
}

__device__ __forceinline__ long long outbox_count(const Outbox& ob) {
    const unsigned long long m = *ob.n;
    return static_cast<long long>(m < static_cast<unsigned long long>(ob.cap) ? m : ob.cap);
}

// Sub-domain k = blockIdx.y takes the particles that left k - 1 upwards and
// k + 1 downwards into its slots after the last one (the step's injection is
// already committed there).
template <class Pos, class Mom>
__global__ void dom_append_kernel(const DomDev* d, int n) {
    const int k = blockIdx.y;
    const DomDev& dst = d[k];
    const long long m1 = k > 0 ? outbox_count(d[k - 1].up) : 0;
    const long long m2 = k + 1 < n ? outbox_count(d[k + 1].down) : 0;
    const long long base = dst.st->n_slots;
    long long room = dst.capacity - base;
    room = room > 0 ? room : 0;
    const long long m = m1 + m2 < room ? m1 + m2 : room;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const Outbox& src = i < m1 ? d[k - 1].up : d[k + 1].down;
        const long long j = i < m1 ? i : i - m1;
        static_cast<Pos*>(dst.xi)[base + i] = static_cast<const Pos*>(src.x)[j];
        static_cast<Mom*>(dst.u)[base + i] = static_cast<const Mom*>(src.u)[j];
        if (dst.ids) dst.ids[base + i] = src.ids ? src.ids[j] : -1;
    }
}

// Counters after the hand-off (one thread): every sub-domain gains the
// particles it took (all of them unless its slots ran out: SCLF_FLAG_CAPACITY)
// and loses the ones it sent; the outboxes are emptied. moved[0] counts the
// particles handed over since creation.
__global__ void dom_commit_kernel(const DomDev* d, int n, unsigned long long* moved) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    long long taken[kMaxDomains];
    for (int k = 0; k < n; ++k) {
        const long long m1 = k > 0 ? outbox_count(d[k - 1].up) : 0;
        const long long m2 = k + 1 < n ? outbox_count(d[k + 1].down) : 0;
        long long room = d[k].capacity - d[k].st->n_slots;
        room = room > 0 ? room : 0;
        taken[k] = m1 + m2 < room ? m1 + m2 : room;
        if (taken[k] < m1 + m2) d[k].st->flags |= SCLF_FLAG_CAPACITY;
    }
    unsigned long long total = 0;
    for (int k = 0; k < n; ++k) {
        DevState* st = d[k].st;
        const long long out = static_cast<long long>(*d[k].down.n + *d[k].up.n);
        st->n_slots += taken[k];
        st->n_live += taken[k] - out;
        total += static_cast<unsigned long long>(taken[k]);
    }
    for (int k = 0; k < n; ++k) {
        *d[k].down.n = 0;
        *d[k].up.n = 0;
    }
    moved[0] += total;
}

}  // namespace
}  // namespace sclf

using namespace sclf;

struct sclf_dtube {
    tube_params p{};
    tube_derived d{};
    int n = 0;
    std::vector<int> cuts;
    std::vector<tube_t> dom;
    std::vector<cudaStream_t> streams;     // one per sub-domain
    cudaStream_t xs = nullptr;             // exchange kernels
    std::vector<cudaEvent_t> ev_dom;       // per sub-domain: end of its kernel phase
    cudaEvent_t ev_x = nullptr;            // end of an exchange phase
    char* mem = nullptr;                   // outboxes, counters, descriptors
    DomDev* dev = nullptr;                 // n descriptors (device)
    unsigned long long* counters = nullptr;  // 2 per sub-domain, then the moved total
    long long ob_cap = 0;
    int64_t host_step = 0;
    int steps_since_compact = 0;
    int compact_every = 64;
    int64_t part_bytes = 0;                // bytes per handed-over particle
    int64_t halo_bytes = 0;                // field bytes exchanged per step
    cudaGraphExec_t chunk = nullptr;       // compact_every steps, captured once
};

namespace sclf {
namespace {

int dt_fail(sclf_dtube* D, int code);

cudaError_t launch_exchange_halo(sclf_dtube* D, int po) {
    const int nb = (D->n + 63) / 64;
    if (D->p.precision == SCLF_FP64)
        dom_halo_kernel<double><<<nb, 64, 0, D->xs>>>(D->dev, D->n, po);
    else
        dom_halo_kernel<float><<<nb, 64, 0, D->xs>>>(D->dev, D->n, po);
    return cudaGetLastError();
}

cudaError_t launch_handoff(sclf_dtube* D) {
    const dim3 grid(64, D->n);
    if (D->p.precision == SCLF_FP64)
        dom_append_kernel<double, double><<<grid, 256, 0, D->xs>>>(D->dev, D->n);
    else if (D->p.precision == SCLF_FIX32)
        dom_append_kernel<int, float><<<grid, 256, 0, D->xs>>>(D->dev, D->n);
    else
        dom_append_kernel<float, float><<<grid, 256, 0, D->xs>>>(D->dev, D->n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dom_commit_kernel<<<1, 1, 0, D->xs>>>(D->dev, D->n, D->counters + 2 * D->n);
    return cudaGetLastError();
}

// The exchange stream waits for every sub-domain's last kernel; then every
// sub-domain's stream waits for the exchange.
int join_domains(sclf_dtube* D) {
    for (int k = 0; k < D->n; ++k) {
        CK(cudaEventRecord(D->ev_dom[k], D->streams[k]));
        CK(cudaStreamWaitEvent(D->xs, D->ev_dom[k], 0));
    }
    return SCLF_OK;
}
int release_domains(sclf_dtube* D) {
    CK(cudaEventRecord(D->ev_x, D->xs));
    for (int k = 0; k < D->n; ++k) CK(cudaStreamWaitEvent(D->streams[k], D->ev_x, 0));
    return SCLF_OK;
}

int dstep(sclf_dtube* D) {
    const int parity = static_cast<int>(D->host_step & 1);
    for (int k = 0; k < D->n; ++k) CK(enqueue_push(D->dom[k], D->streams[k]));
    int rc = join_domains(D);
    if (rc) return rc;
    dom_current_kernel<<<(D->n + 63) / 64, 64, 0, D->xs>>>(D->dev, D->n);
    CK(cudaGetLastError());
    rc = release_domains(D);
    if (rc) return rc;
    for (int k = 0; k < D->n; ++k) CK(enqueue_field(D->dom[k], parity, D->streams[k]));
    rc = join_domains(D);
    if (rc) return rc;
    CK(launch_handoff(D));
    CK(launch_exchange_halo(D, parity ^ 1));
    rc = release_domains(D);
    if (rc) return rc;
    D->host_step += 1;
    for (int k = 0; k < D->n; ++k) {
        D->dom[k]->host_step += 1;
        D->dom[k]->steps_since_compact = 0;
    }
    if (++D->steps_since_compact >= D->compact_every) {
        for (int k = 0; k < D->n; ++k) CK(enqueue_compact(D->dom[k], D->streams[k], 0));
        rc = join_domains(D);
        if (rc) return rc;
        rc = release_domains(D);
        if (rc) return rc;
        D->steps_since_compact = 0;
    }
    return SCLF_OK;
}

// compact_every steps from an even step right after a compaction check,
// captured once from the exchange stream (the sub-domain streams join the
// capture through its event and rejoin it at the end; the events between the
// streams become graph edges) and replayed by dtube_run. The host's step
// counters are restored after the capture and advanced per replay.
int capture_dchunk(sclf_dtube* D) {
    const int64_t hs = D->host_step;
    std::vector<int64_t> ths(D->n);
    for (int k = 0; k < D->n; ++k) ths[k] = D->dom[k]->host_step;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(D->xs, cudaStreamCaptureModeThreadLocal));
    int rc = release_domains(D);
    for (int s = 0; s < D->compact_every && rc == SCLF_OK; ++s) rc = dstep(D);
    if (rc == SCLF_OK) rc = join_domains(D);
    const cudaError_t e2 = cudaStreamEndCapture(D->xs, &g);
    D->host_step = hs;
    for (int k = 0; k < D->n; ++k) {
        D->dom[k]->host_step = ths[k];
        D->dom[k]->steps_since_compact = 0;
    }
    D->steps_since_compact = 0;
    if (rc != SCLF_OK || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc != SCLF_OK ? rc : cuda_fail(e2);
    }
    const cudaError_t e = cudaGraphInstantiate(&D->chunk, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return SCLF_OK;
}

int launch_dchunk(sclf_dtube* D) {
    int rc = join_domains(D);
    if (rc) return rc;
    CK(cudaGraphLaunch(D->chunk, D->xs));
    rc = release_domains(D);
    if (rc) return rc;
    D->host_step += D->compact_every;
    for (int k = 0; k < D->n; ++k) {
        D->dom[k]->host_step += D->compact_every;
        D->dom[k]->steps_since_compact = 0;
    }
    D->steps_since_compact = 0;
    return SCLF_OK;
}

int sync_all(sclf_dtube* D) {
    for (int k = 0; k < D->n; ++k) CK(cudaStreamSynchronize(D->streams[k]));
    CK(cudaStreamSynchronize(D->xs));
    return SCLF_OK;
}

// Only the base sub-domain injects: the others' pending count is zero.
int clear_injection(sclf_dtube* D) {
    for (int k = 1; k < D->n; ++k) {
        sclf_tube* t = D->dom[k];
        CK(cudaMemsetAsync(&t->st->n_inj, 0, sizeof(long long), t->stream));
        CK(cudaMemsetAsync(&t->st->surface_field, 0, sizeof(double), t->stream));
    }
    return sync_all(D);
}

void destroy(sclf_dtube* D) {
    if (D->chunk) cudaGraphExecDestroy(D->chunk);
    for (tube_t t : D->dom)
        if (t) {
            t->owned = false;
            tube_destroy(t);
        }
    if (D->mem) cudaFree(D->mem);
    for (cudaEvent_t e : D->ev_dom)
        if (e) cudaEventDestroy(e);
    if (D->ev_x) cudaEventDestroy(D->ev_x);
    for (cudaStream_t s : D->streams)
        if (s) cudaStreamDestroy(s);
    if (D->xs) cudaStreamDestroy(D->xs);
    delete D;
}

int dt_fail(sclf_dtube* D, int code) {
    destroy(D);
    return code;
}

}  // namespace
}  // namespace sclf

extern "C" {

int dtube_create(const tube_params* p, int32_t n, const int64_t* cuts, dtube_t* out) {
    if (!p || !out || n < 1 || n > kMaxDomains) return SCLF_EINVAL;
    *out = nullptr;
    tube_derived d;
    int rc = tube_derive(p, &d);
    if (rc) return rc;
    if (p->accumulate != SCLF_ACC_FIXED64) return SCLF_EINVAL;
    const int64_t nz = p->Nz;
    std::vector<int> c(n + 1);
    for (int k = 0; k <= n; ++k) {
        const int64_t v = cuts ? cuts[k] : (nz * k) / n;
        c[k] = static_cast<int>(v);
        if (v < 0 || v > nz) return SCLF_EINVAL;
    }
    if (c[0] != 0 || c[n] != nz) return SCLF_EINVAL;
    for (int k = 0; k < n; ++k)
        if (c[k + 1] - c[k] < 2) return SCLF_EINVAL;

    sclf_dtube* D = new (std::nothrow) sclf_dtube();
    if (!D) return SCLF_ENOMEM;
    D->p = *p;
    D->p.rho_gj_user = nullptr;
    D->d = d;
    D->n = n;
    D->cuts = c;
    D->compact_every = p->compact_interval > 0 ? p->compact_interval : 64;
    D->streams.assign(n, nullptr);
    D->ev_dom.assign(n, nullptr);
    D->dom.assign(n, nullptr);
    if (cudaStreamCreateWithFlags(&D->xs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->ev_x, cudaEventDisableTiming) != cudaSuccess)
        return dt_fail(D, SCLF_ECUDA);
    for (int k = 0; k < n; ++k) {
        if (cudaStreamCreateWithFlags(&D->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&D->ev_dom[k], cudaEventDisableTiming) != cudaSuccess)
            return dt_fail(D, SCLF_ECUDA);
        tube_params q = *p;
        q.use_graphs = 0;
        rc = tube_create(&q, nullptr, 0, D->streams[k], &D->dom[k]);
        if (rc) return dt_fail(D, rc);
        D->dom[k]->owned = true;
        D->dom[k]->dom_lo = c[k];
        D->dom[k]->dom_hi = c[k + 1];
    }
    // outboxes (two per sub-domain), their counters and the descriptors
    const int64_t rs = p->precision == SCLF_FP64 ? 8 : 4;
    const bool ids = p->track_ids != 0;
    D->ob_cap = std::max<long long>(65536, p->capacity / 8);
    D->part_bytes = 2 * rs + (ids ? 8 : 0);
    const int64_t box = (D->ob_cap * D->part_bytes + 255) / 256 * 256;
    const int64_t cnt_bytes = (int64_t(2 * n + 1) * 8 + 255) / 256 * 256;
    const int64_t desc_bytes = (int64_t(n) * sizeof(DomDev) + 255) / 256 * 256;
    const int64_t pair_bytes = int64_t(n) * 2 * sizeof(Outbox);
    if (cudaMalloc(&D->mem, 2 * n * box + cnt_bytes + desc_bytes + pair_bytes) != cudaSuccess) {
        D->mem = nullptr;
        return dt_fail(D, SCLF_ENOMEM);
    }
    D->counters = reinterpret_cast<unsigned long long*>(D->mem + 2 * n * box);
    D->dev = reinterpret_cast<DomDev*>(D->mem + 2 * n * box + cnt_bytes);
    Outbox* pairs = reinterpret_cast<Outbox*>(D->mem + 2 * n * box + cnt_bytes + desc_bytes);
    std::vector<Outbox> hpairs(2 * n);
    if (cudaMemset(D->counters, 0, cnt_bytes) != cudaSuccess) return dt_fail(D, SCLF_ECUDA);
    std::vector<DomDev> h(n);
    for (int k = 0; k < n; ++k) {
        sclf_tube* t = D->dom[k];
        for (int side = 0; side < 2; ++side) {
            char* b = D->mem + (2 * k + side) * box;
            Outbox ob;
            ob.x = b;
            ob.u = b + D->ob_cap * rs;
            ob.ids = ids ? reinterpret_cast<long long*>(b + 2 * D->ob_cap * rs) : nullptr;
            ob.n = D->counters + 2 * k + side;
            ob.cap = D->ob_cap;
            (side == 0 ? t->out_down : t->out_up) = ob;
        }
        DomDev& dd = h[k];
        dd.st = t->st;
        dd.xi = t->xi;
        dd.u = t->u;
        dd.ids = t->ids;
        dd.jacc = static_cast<long long*>(t->jacc);
        dd.ez = t->ez;
        dd.b[0] = t->b[0];
        dd.b[1] = t->b[1];
        dd.ez2 = t->ez2;
        dd.capacity = t->p.capacity;
        dd.lo = c[k];
        dd.hi = c[k + 1];
        dd.down = t->out_down;
        dd.up = t->out_up;
        hpairs[2 * k] = t->out_down;
        hpairs[2 * k + 1] = t->out_up;
        t->out_dev = pairs + 2 * k;                  // the particle kernels read them there
    }
    if (cudaMemcpy(D->dev, h.data(), int64_t(n) * sizeof(DomDev), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(pairs, hpairs.data(), pair_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return dt_fail(D, SCLF_ECUDA);
    // per boundary and step: J of two cells, B_phi of two cells, two E_z table entries
    const int64_t ts = p->precision == SCLF_FP64 ? 8 : 4;
    D->halo_bytes = int64_t(n - 1) * (2 * 8 + 2 * 8 + 2 * ts);
    rc = clear_injection(D);
    if (rc) return dt_fail(D, rc);
    *out = D;
    return SCLF_OK;
}

int dtube_destroy(dtube_t dt) {
    if (!dt) return SCLF_EINVAL;
    sync_all(dt);
    destroy(dt);
    return SCLF_OK;
}

int dtube_domains(dtube_t dt, int32_t* n) {
    if (!dt || !n) return SCLF_EINVAL;
    *n = dt->n;
    return SCLF_OK;
}

int dtube_domain(dtube_t dt, int32_t i, tube_t* tube, int64_t* lo, int64_t* hi) {
    if (!dt || i < 0 || i >= dt->n) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    if (tube) *tube = dt->dom[i];
    if (lo) *lo = dt->cuts[i];
    if (hi) *hi = dt->cuts[i + 1];
    return SCLF_OK;
}

int dtube_load_particles(dtube_t dt, int64_t n, const double* z, const double* u) {
    NvtxRange nvtx_range("dtube_load_particles");
    if (!dt || n < 0 || (n > 0 && (!z || !u))) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    for (tube_t t : dt->dom) {
        DevState h;
        rc = read_state(t, &h);
        if (rc) return rc;
        if (h.n_slots != 0 || h.step != 0 || h.total_injected != 0) return SCLF_ESTATE;
    }
    sclf_tube* t0 = dt->dom[0];
    std::vector<char> xs, us;
    rc = native_particles(t0, n, z, u, xs, us);
    if (rc) return rc;
    const int64_t rs = dt->p.precision == SCLF_FP64 ? 8 : 4;
    std::vector<std::vector<char>> px(dt->n), pu(dt->n);
    std::vector<std::vector<int64_t>> pid(dt->n);
    for (int64_t i = 0; i < n; ++i) {
        const double cell = raw_cells(t0, xs.data(), i);
        const int k = static_cast<int>(std::upper_bound(dt->cuts.begin() + 1, dt->cuts.end(),
                                                        static_cast<int>(cell)) -
                                       (dt->cuts.begin() + 1));
        px[k].insert(px[k].end(), xs.data() + i * rs, xs.data() + (i + 1) * rs);
        pu[k].insert(pu[k].end(), us.data() + i * rs, us.data() + (i + 1) * rs);
        pid[k].push_back(i);
    }
    for (int k = 0; k < dt->n; ++k) {
        const int64_t m = static_cast<int64_t>(pid[k].size());
        if (m > dt->dom[k]->p.capacity) return SCLF_ECAPACITY;
        rc = append_raw(dt->dom[k], m, px[k].data(), pu[k].data(),
                        dt->dom[k]->ids ? pid[k].data() : nullptr);
        if (rc) return rc;
    }
    // IDs continue after the n loaded ones in the base sub-domain, which injects
    long long tot = n;
    CK(cudaMemcpyAsync(&t0->st->total_injected, &tot, sizeof(long long), cudaMemcpyHostToDevice,
                       t0->stream));
    return clear_injection(dt);
}

int dtube_set_fields(dtube_t dt, const double* Ez, const double* Er, const double* Bphi) {
    if (!dt || !Ez || !Er) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    for (tube_t t : dt->dom) {
        rc = set_fields_host(t, Ez, Er, Bphi);
        if (rc) return rc;
    }
    return clear_injection(dt);
}

int dtube_solve_fields(dtube_t dt) {
    NvtxRange nvtx_range("dtube_solve_fields");
    if (!dt) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    const int64_t nz = dt->p.Nz;
    std::vector<double> rho(nz + 1, 0.0), part(nz + 1), src(nz + 1), phi(nz + 1), ez0(nz);
    for (tube_t t : dt->dom) {
        rc = tube_read_fields(t, nullptr, nullptr, nullptr, nullptr, part.data());
        if (rc) return rc;
        for (int64_t j = 0; j <= nz; ++j) rho[j] += part[j];
    }
    const std::vector<double>& rho_gj = dt->dom[0]->rho_gj;
    for (int64_t j = 0; j <= nz; ++j) src[j] = rho_gj[j] - rho[j];
    solve_poisson(src.data(), nz, dt->d.dz, phi.data());
    for (int64_t j = 0; j < nz; ++j) ez0[j] = -(phi[j + 1] - phi[j]) / dt->d.dz;
    return dtube_set_fields(dt, ez0.data(), phi.data(), nullptr);
}

int dtube_step(dtube_t dt) {
    NvtxRange nvtx_range("dtube_step");
    if (!dt) return SCLF_EINVAL;
    return dstep(dt);
}

int dtube_run(dtube_t dt, int64_t nsteps) {
    NvtxRange nvtx_range("dtube_run");
    if (!dt || nsteps < 0) return SCLF_EINVAL;
    sclf_dtube* D = dt;
    while (nsteps > 0) {
        int rc;
        if (D->p.use_graphs && D->compact_every % 2 == 0 && (D->host_step & 1) == 0 &&
            D->steps_since_compact == 0 && nsteps >= D->compact_every) {
            if (!D->chunk && (rc = capture_dchunk(D)) != SCLF_OK) return rc;
            if ((rc = launch_dchunk(D)) != SCLF_OK) return rc;
            nsteps -= D->compact_every;
            continue;
        }
        if ((rc = dstep(D)) != SCLF_OK) return rc;
        nsteps -= 1;
    }
    return SCLF_OK;
}

int dtube_status(dtube_t dt, tube_stats* out) {
    if (!dt || !out) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    for (int k = 0; k < dt->n; ++k) {
        DevState h;
        rc = read_state(dt->dom[k], &h);
        if (rc) return rc;
        out->n_particles += h.n_live;
        out->n_slots += h.n_slots;
        out->last_removed += h.last_removed;
        out->flags |= h.flags;
        if (k == 0) {
            out->step = h.step;
            out->total_injected = h.total_injected;
            out->last_injected = h.last_injected;
            out->pending_injection = h.n_inj;
            out->surface_field = h.surface_field;
        }
    }
    return SCLF_OK;
}

int dtube_read_fields(dtube_t dt, double* Ez, double* Er, double* Bphi, double* J) {
    if (!dt) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    const int64_t nz = dt->p.Nz;
    std::vector<double> ez(nz), er(nz + 1), b(nz), j(nz);
    for (int k = 0; k < dt->n; ++k) {
        rc = tube_read_fields(dt->dom[k], ez.data(), er.data(), b.data(), j.data(), nullptr);
        if (rc) return rc;
        const int lo = dt->cuts[k], hi = dt->cuts[k + 1];
        const int hi_node = k + 1 == dt->n ? hi + 1 : hi;
        if (Ez) std::copy(ez.begin() + lo, ez.begin() + hi, Ez + lo);
        if (Bphi) std::copy(b.begin() + lo, b.begin() + hi, Bphi + lo);
        if (J) std::copy(j.begin() + lo, j.begin() + hi, J + lo);
        if (Er) std::copy(er.begin() + lo, er.begin() + hi_node, Er + lo);
    }
    return SCLF_OK;
}

int dtube_exchange_stats(dtube_t dt, int64_t* steps, int64_t* field_bytes, int64_t* particles,
                         int64_t* particle_bytes) {
    if (!dt) return SCLF_EINVAL;
    int rc = sync_all(dt);
    if (rc) return rc;
    unsigned long long moved = 0;
    CK(cudaMemcpy(&moved, dt->counters + 2 * dt->n, sizeof(moved), cudaMemcpyDeviceToHost));
    if (steps) *steps = dt->host_step;
    if (field_bytes) *field_bytes = dt->host_step * dt->halo_bytes;
    if (particles) *particles = static_cast<int64_t>(moved);
    if (particle_bytes) *particle_bytes = static_cast<int64_t>(moved) * dt->part_bytes;
    return SCLF_OK;
}

}  // extern "C"
