// tube_push_deposit_static: one gather-push-deposit pass over caller-owned
// FP32 particles that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose own allocator
// has reserved the device's memory up front, a plug-in whose host forbids
// allocation once it is running, or a latency-critical loop where the
// implicit device-wide synchronisation of cudaMalloc/cudaFree would stall
// other work. This entry point serves them. Its scratch (the fixed-point
// current sums, the float32 gather table and a removal counter) lives in
// one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits (about 1 MB). The caller still
// provides the particles, the E_z grid and the outputs.
//
// The arithmetic is the same as one pass of the tube step without injection:
// cloud-in-cell gather of E_z, the Eq. 1 push (q/m = -1, c = 1), the
// charge-conserving current deposit summed in 2^-32 fixed point (each F_j
// quantised before differencing), and removal
// of particles that leave [0, Nz) (their slot becomes a hole, xi = -1).
//
// CUDA loads modules lazily by default, and loading this file's module (its
// kernels and the scratch array) takes device memory. The per-device set-up
// below therefore does all of that loading at once, on the first call on a
// device: that call may allocate, every later call allocates nothing.
#include <mutex>

#include "sclf_internal.h"

namespace {

constexpr int kMaxNz = SCLF_STATIC_MAX_NZ;
constexpr int kMaxDevices = 64;

struct StaticScratch {
    unsigned long long acc[kMaxNz];          // fixed-point current sums, 2^-32 units
    float table[2 * (kMaxNz + 1)];           // (E_{m-1/2}, E_{m+1/2}) per node m
    unsigned long long removed;              // particles removed by this call
    unsigned int nonfinite;                  // 1 if a particle's push gave NaN/Inf
    unsigned int pad0;
    unsigned long long pad[30];
};

// The only scratch of this entry point. In host code the name is a host-side
// stand-in, not a device address: host code uses the address from
// cudaGetSymbolAddress (scratch_on_current_device) and passes it on.
static __device__ __align__(256) StaticScratch g_static_scratch;

__global__ void static_clear(StaticScratch* sc, int nz) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nz; j += gridDim.x * blockDim.x)
        sc->acc[j] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->removed = 0ull;
        sc->nonfinite = 0u;
    }
}

__global__ void static_table(StaticScratch* sc, const double* ez, int nz) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > nz) return;
    const int lo = m - 1 < 0 ? 0 : m - 1;
    const int hi = m > nz - 1 ? nz - 1 : m;
    sc->table[2 * m] = static_cast<float>(ez[lo]);
    sc->table[2 * m + 1] = static_cast<float>(ez[hi]);
}

__device__ __forceinline__ float clamp01f(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

// F = clamp(v, 0, 1) in 2^-32 units, rounded half-even (as in the tube step:
// each F is quantised before the difference F_j(x1) - F_j(x0) is taken).
__device__ __forceinline__ long long qfrac(float v) {
    v = clamp01f(v);
    return v >= 1.0f ? (1LL << 32) : static_cast<long long>(__float2uint_rn(v * 4294967296.0f));
}

__global__ void static_push(StaticScratch* sc, float* xi, float* u, long long n, int nz,
                            float nzf, float dt, float cfl) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float x = xi[i];
        if (!(x >= 0.0f && x < nzf)) continue;                 // hole
        const float h = x + 0.5f;
        const float mf = floorf(h);
        const float f = h - mf;
        int m = static_cast<int>(mf);
        m = m < 0 ? 0 : (m > nz ? nz : m);
        const float ep = (1.0f - f) * sc->table[2 * m] + f * sc->table[2 * m + 1];
        const float u1 = u[i] - ep * dt;
        const float g = sqrtf(1.0f + u1 * u1);
        const float x1 = x + (u1 / g) * cfl;
        if (!(isfinite(x1) && isfinite(u1))) {
            xi[i] = -1.0f;
            u[i] = 0.0f;
            atomicAdd(&sc->removed, 1ull);
            sc->nonfinite = 1u;
            continue;
        }
        const int c0 = static_cast<int>(floorf(x));
        const int c1 = static_cast<int>(floorf(x1));
        {
            const float jf = static_cast<float>(c0);
            const long long q = qfrac(x1 - jf) - qfrac(x - jf);
            if (q) atomicAdd(&sc->acc[c0], static_cast<unsigned long long>(q));
        }
        if (c1 != c0 && c1 >= 0 && c1 < nz) {
            const float jf = static_cast<float>(c1);
            const long long q = qfrac(x1 - jf) - qfrac(x - jf);
            if (q) atomicAdd(&sc->acc[c1], static_cast<unsigned long long>(q));
        }
        if (x1 >= 0.0f && x1 < nzf) {
            xi[i] = x1;
            u[i] = u1;
        } else {
            xi[i] = -1.0f;
            u[i] = 0.0f;
            atomicAdd(&sc->removed, 1ull);
        }
    }
}

__global__ void static_finish(const StaticScratch* sc, int nz, double s_over_dt, double* j_out,
                              long long* n_removed, unsigned int* flags) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nz; j += gridDim.x * blockDim.x) {
        const double ssum = double(static_cast<long long>(sc->acc[j])) * sclf::kFixedInv;
        j_out[j] = s_over_dt * ssum;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (n_removed) *n_removed = static_cast<long long>(sc->removed);
        if (flags && sc->nonfinite) *flags |= SCLF_FLAG_NONFINITE;
    }
}

std::mutex g_mu;
StaticScratch* g_ptr[kMaxDevices] = {};

// Set-up, once per device, with that device current: load the module's four
// kernels (cudaFuncGetAttributes loads a kernel that has not been loaded
// yet) and look up the device address of the scratch array, so that no
// later call loads anything. A cudaDeviceReset invalidates the cached
// address; the library must then be reloaded before this entry point is
// used again on that device.
int scratch_on_current_device(StaticScratch** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCLF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SCLF_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, static_clear) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, static_table) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, static_push) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, static_finish) != cudaSuccess)
            return SCLF_ECUDA;
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) return SCLF_ECUDA;
        g_ptr[dev] = static_cast<StaticScratch*>(p);
    }
    *out = g_ptr[dev];
    return SCLF_OK;
}

}  // namespace

extern "C" int tube_push_deposit_static(float* xi, float* u, int64_t n, const double* ez,
                                        int32_t nz, double dt, double dz, double s,
                                        double* j_out, int64_t* n_removed, uint32_t* flags,
                                        void* stream) {
    if (nz < 2 || nz > kMaxNz) return SCLF_EINVAL;             // beyond the static scratch
    if (n < 0 || (n > 0 && (!xi || !u)) || !ez || !j_out) return SCLF_EINVAL;
    if (!(dt > 0.0 && dz > 0.0 && dt < dz) || !(s < 0.0)) return SCLF_EINVAL;
    // an error the caller's own work left pending is not this call's: refuse
    // to launch, and leave it pending for the caller
    if (cudaPeekAtLastError() != cudaSuccess) return SCLF_ECUDA;
    StaticScratch* sc = nullptr;
    const int rc = scratch_on_current_device(&sc);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int gz = (nz + 255) / 256;
    static_clear<<<gz, 256, 0, st>>>(sc, nz);
    static_table<<<(nz + 1 + 255) / 256, 256, 0, st>>>(sc, ez, nz);
    if (n > 0) {
        long long g = (n + 255) / 256;
        if (g > 4096) g = 4096;
        static_push<<<static_cast<int>(g), 256, 0, st>>>(
            sc, xi, u, n, nz, static_cast<float>(nz), static_cast<float>(dt),
            static_cast<float>(dt / dz));
    }
    static_finish<<<gz, 256, 0, st>>>(sc, nz, s / dt, j_out,
                                      reinterpret_cast<long long*>(n_removed), flags);
    return cudaGetLastError() == cudaSuccess ? SCLF_OK : SCLF_ECUDA;
}
