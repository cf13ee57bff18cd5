// fre_moments_noalloc: the conservation sums and droplet moments of the
// observables, computed from caller-owned device populations without any
// device allocation.  The per-block partial sums live in a file-scope
// __device__ array instead of context memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fre_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 512;                          // blocks of each reduction pass
constexpr int kPass1 = 8;                                // rho, phi, volume, W, count, Wx, Wy, Wz
constexpr int kPass2 = 6;                                // central second moments
constexpr int kScratchDoubles = kMaxBlocks * (kPass1 + kPass2) + 32;  // 57,600 B
constexpr long long kMaxNodes = 1LL << 30;

// Shared by every call on a device; holds the last call's partials.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch, looked up once per CUDA context.  The
// address belongs to the module loaded into a context: after a
// cudaDeviceReset, or with another context current, the module may sit
// elsewhere, so the cache is keyed on the context's unique id (never reused
// within a process), not on the device index.
struct ScratchAddr {
    unsigned long long ctx_id;
    double *ptr;
};
constexpr int kMaxContexts = 64;
ScratchAddr g_scratch_addr[kMaxContexts] = {};
int g_scratch_n = 0, g_scratch_next = 0;
std::mutex g_setup_mutex;

// Driver entry points for the id of the current context, resolved through
// the runtime (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the context current on this thread; false if there is none yet.
// Called with g_setup_mutex held.
bool current_context_id(unsigned long long *id) {
    static bool resolved = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!resolved) {
        resolved = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
    }
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}


__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int NV>
__device__ __forceinline__ void block_store(const double *v, double *out) {
    __shared__ double sh[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double r = warp_sum_d(v[k]);
        if (lane == 0) sh[wid][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += sh[w][threadIdx.x];
        out[blockIdx.x * NV + threadIdx.x] = acc;
    }
}

// Pass 1: rho = sum f_i, phi = sum g_i at every node; the sums of rho, phi,
// (1 + phi)/2 and, over phi > 0, of w = (1 + phi)/2 and w x, w y, w z.
template <int Q>
__global__ void __launch_bounds__(kThreads) k_na_pass1(const double *__restrict__ f, const double *__restrict__ g,
                                                      int nx, int ny, long long n, double *scratch) {
    double v[kPass1] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double rho = 0.0, ph = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rho += f[(size_t)i * n + k];
            ph += g[(size_t)i * n + k];
        }
        v[0] += rho;
        v[1] += ph;
        v[2] += 0.5 * (1.0 + ph);
        if (ph > 0.0) {
            const double w = 0.5 * (1.0 + ph);
            const long long r = k % ((long long)nx * ny);
            v[3] += w;
            v[4] += 1.0;
            v[5] += w * (double)(r % nx);
            v[6] += w * (double)(r / nx);
            v[7] += w * (double)(k / ((long long)nx * ny));
        }
    }
    block_store<kPass1>(v, scratch);
}

// Sum the pass-1 partials in block order, then pass 2: central second
// moments about the centroid.
template <int Q>
__global__ void __launch_bounds__(kThreads) k_na_pass2(const double *__restrict__ g, int nx, int ny, long long n,
                                                      int nblocks, double *scratch) {
    __shared__ double tot[kPass1];
    if (threadIdx.x < kPass1) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += scratch[b * kPass1 + threadIdx.x];
        tot[threadIdx.x] = acc;
    }
    __syncthreads();
    const double W = tot[3];
    const double X = W > 0 ? tot[5] / W : 0.0, Y = W > 0 ? tot[6] / W : 0.0, Z = W > 0 ? tot[7] / W : 0.0;
    double v[kPass2] = {0, 0, 0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double ph = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) ph += g[(size_t)i * n + k];
        if (!(ph > 0.0)) continue;
        const double w = 0.5 * (1.0 + ph);
        const long long r = k % ((long long)nx * ny);
        const double dx = (double)(r % nx) - X, dy = (double)(r / nx) - Y,
                     dz = (double)(k / ((long long)nx * ny)) - Z;
        v[0] += w * dx * dx;
        v[1] += w * dy * dy;
        v[2] += w * dz * dz;
        v[3] += w * dx * dy;
        v[4] += w * dx * dz;
        v[5] += w * dy * dz;
    }
    block_store<kPass2>(v, scratch + kMaxBlocks * kPass1);
}

// Totals in block order and the derived quantities into out[16].
__global__ void k_na_final(int nblocks, const double *scratch, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t1[kPass1], t2[kPass2];
    for (int k = 0; k < kPass1; ++k) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += scratch[b * kPass1 + k];
        t1[k] = acc;
    }
    for (int k = 0; k < kPass2; ++k) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += scratch[kMaxBlocks * kPass1 + b * kPass2 + k];
        t2[k] = acc;
    }
    const double W = t1[3];
    for (int k = 0; k < 5; ++k) out[k] = t1[k];
    for (int k = 5; k < 16; ++k) out[k] = 0.0;
    if (W > 0.0) {
        for (int k = 0; k < 3; ++k) out[5 + k] = t1[5 + k] / W;
        for (int k = 0; k < 6; ++k) out[8 + k] = t2[k] / W;
        const double a = out[8], b = out[9], c = out[11];
        const double m = 0.5 * (a + b), r = sqrt(0.25 * (a - b) * (a - b) + c * c);
        double l1 = m + r, l2 = m - r;
        if (l2 < 0.0) l2 = 0.0;
        const double s1 = sqrt(l1), s2 = sqrt(l2);
        out[14] = (s1 + s2) > 0.0 ? (s1 - s2) / (s1 + s2) : 0.0;
        out[15] = 0.5 * atan2(2.0 * c, a - b) * (180.0 / 3.14159265358979323846);
    }
}

fre_status na_fail(fre_status s, const char *msg) {
    fre::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" {

fre_status fre_moments_noalloc(int lattice, int nx, int ny, int nz, const double *f_dev, const double *g_dev,
                               double *out_dev, void *cuda_stream) {
    if (lattice != FRE_D2Q9 && lattice != FRE_D3Q19) return na_fail(FRE_ERR_ARG, "fre_moments_noalloc: unknown lattice");
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == FRE_D2Q9 && nz != 1))
        return na_fail(FRE_ERR_ARG, "fre_moments_noalloc: sizes must be >= 1 (nz = 1 for D2Q9)");
    const long long n = (long long)nx * ny * nz;
    if (n > kMaxNodes)
        return na_fail(FRE_ERR_ARG, "fre_moments_noalloc: more than 2^30 nodes (the largest lattice it accepts)");
    if (!f_dev || !g_dev || !out_dev) return na_fail(FRE_ERR_ARG, "fre_moments_noalloc: NULL pointer");

    double *scratch = nullptr;
    {
        // first call in a context: look up the device address of the
        // file-scope scratch array (the host-side symbol is not an address a
        // kernel may use); cudaGetSymbolAddress also makes the device's
        // primary context current if no context is current yet
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        unsigned long long id = 0;
        bool have_id = current_context_id(&id);
        for (int k = 0; have_id && k < g_scratch_n; ++k)
            if (g_scratch_addr[k].ctx_id == id) scratch = g_scratch_addr[k].ptr;
        if (!scratch) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                char msg[256];
                snprintf(msg, sizeof(msg), "fre_moments_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return na_fail(FRE_ERR_CUDA, msg);
            }
            scratch = static_cast<double *>(p);
            if (!have_id) have_id = current_context_id(&id);
            if (have_id) {
                g_scratch_addr[g_scratch_next] = {id, scratch};
                g_scratch_next = (g_scratch_next + 1) % kMaxContexts;
                if (g_scratch_n < kMaxContexts) ++g_scratch_n;
            }
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    long long nb = (n + kThreads - 1) / kThreads;
    const int nblocks = (int)(nb < kMaxBlocks ? nb : kMaxBlocks);
    if (lattice == FRE_D2Q9) {
        k_na_pass1<9><<<nblocks, kThreads, 0, st>>>(f_dev, g_dev, nx, ny, n, scratch);
        k_na_pass2<9><<<nblocks, kThreads, 0, st>>>(g_dev, nx, ny, n, nblocks, scratch);
    } else {
        k_na_pass1<19><<<nblocks, kThreads, 0, st>>>(f_dev, g_dev, nx, ny, n, scratch);
        k_na_pass2<19><<<nblocks, kThreads, 0, st>>>(g_dev, nx, ny, n, nblocks, scratch);
    }
    k_na_final<<<1, 32, 0, st>>>(nblocks, scratch, out_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "fre_moments_noalloc: launch failed: %s", cudaGetErrorString(e));
        return na_fail(FRE_ERR_CUDA, msg);
    }
    return FRE_OK;
}

}  // extern "C"
