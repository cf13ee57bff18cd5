// Connected components of the droplet phase phi > 0: breakup detection.
//
// A drop that breaks up (Sec. 3: end-pinching, capillary-wave breakup,
// over-stretching in the four-roller device) leaves two or more separate
// drops.  The phase is the set of fluid nodes with phi > 0; two of its nodes
// are connected when a lattice velocity links them (D2Q9: 8 neighbours,
// D3Q19: 18), with the device's periodic wrap (x and z always, y except
// across the shear walls).  Every node of a component gets the component's
// smallest node index as its label.
//
// Labelling by concurrent union-find on the label array itself: every phase
// node starts as its own root; for each link between two phase nodes the
// roots of both ends are found and the larger root is hooked under the
// smaller with a compare-and-swap (retried if another thread hooked it
// first).  A root is only ever hooked under a smaller one, so parents are
// always smaller than their children and the root a component ends with is
// its smallest index, whatever the order the threads ran in: the labels are
// deterministic.  A last pass points every node at its root.
#include <cuda_runtime.h>

#include "fre_ctx.h"
#include "lattice.cuh"

namespace fre {
namespace {

constexpr int kCclThreads = 256;

__device__ __forceinline__ int ld_label(const int *lab, int x) { return *((const volatile int *)lab + x); }

// root of x; halves the path on the way (any ancestor is a valid parent)
__device__ __forceinline__ int ccl_find(int *lab, int x) {
    while (true) {
        const int p = ld_label(lab, x);
        if (p == x) return x;
        const int gp = ld_label(lab, p);
        if (gp != p) *((volatile int *)lab + x) = gp;
        x = gp;
    }
}

__device__ __forceinline__ void ccl_union(int *lab, int a, int b) {
    while (true) {
        a = ccl_find(lab, a);
        b = ccl_find(lab, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        // hook the larger root a under b, unless a stopped being a root
        const int old = atomicCAS(lab + a, a, b);
        if (old == a) return;
        a = old;
    }
}

__device__ __forceinline__ void ccl_coords(const Geo &G, int n, int &x, int &y, int &z) {
    const int nxy = G.nx * G.ny;
    z = n / nxy;
    const int r = n - z * nxy;
    y = r / G.nx;
    x = r - y * G.nx;
}

template <typename T>
__global__ void __launch_bounds__(kCclThreads) k_ccl_init(Geo G, const T *__restrict__ phi, int *lab) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        const bool fluid = G.device != FRE_FOUR_ROLLER || G.solid[n] == 0;
        lab[n] = (fluid && phi[n] > T(0)) ? n : -1;
    }
}

// one link of every opposite pair (i < opp(i)) per phase node
template <int Q>
__global__ void __launch_bounds__(kCclThreads) k_ccl_union(Geo G, int *lab) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < G.n; n += gridDim.x * blockDim.x) {
        if (ld_label(lab, n) < 0) continue;
        int x, y, z;
        ccl_coords(G, n, x, y, z);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (Lat<Q>::opp(i) < i) continue;
            int yn = y + Lat<Q>::cy(i);
            if (G.device == FRE_SHEAR && (yn < 0 || yn >= G.ny)) continue;
            yn = yn < 0 ? yn + G.ny : (yn >= G.ny ? yn - G.ny : yn);
            int xn = x + Lat<Q>::cx(i), zn = z + Lat<Q>::cz(i);
            xn = xn < 0 ? xn + G.nx : (xn >= G.nx ? xn - G.nx : xn);
            zn = zn < 0 ? zn + G.nz : (zn >= G.nz ? zn - G.nz : zn);
            const int m = (zn * G.ny + yn) * G.nx + xn;
            if (ld_label(lab, m) >= 0) ccl_union(lab, n, m);
        }
    }
}

// every phase node points at its root; component sizes at the roots
__global__ void __launch_bounds__(kCclThreads) k_ccl_flatten(long long n_nodes, int *lab, int *sizes) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
        if (ld_label(lab, n) < 0) continue;
        const int r = ccl_find(lab, n);
        lab[n] = r;
        atomicAdd(sizes + r, 1);
    }
}

// roots of the components with at least min_size nodes: (size, root) pairs
__global__ void __launch_bounds__(kCclThreads) k_ccl_roots(long long n_nodes, const int *lab, const int *sizes,
                                                            long long min_size, int cap, int *count,
                                                            long long *pairs) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
        if (lab[n] != n || (long long)sizes[n] < min_size) continue;
        const int k = atomicAdd(count, 1);
        if (k < cap) {
            pairs[2 * k] = sizes[n];
            pairs[2 * k + 1] = n;
        }
    }
}

}  // namespace

void ccl_label(const Launch &L, int lattice, int precision, long long min_size, const CclBuffers &B) {
    const long long n = L.G.n;
    const long long blocks = (n + kCclThreads - 1) / kCclThreads;
    const int g = (int)(blocks < 4096 ? (blocks < 1 ? 1 : blocks) : 4096);
    if (precision == FRE_FP64)
        k_ccl_init<double><<<g, kCclThreads, 0, L.stream>>>(L.G, static_cast<const double *>(L.phi), B.labels);
    else
        k_ccl_init<float><<<g, kCclThreads, 0, L.stream>>>(L.G, static_cast<const float *>(L.phi), B.labels);
    if (lattice == FRE_D2Q9) k_ccl_union<9><<<g, kCclThreads, 0, L.stream>>>(L.G, B.labels);
    else k_ccl_union<19><<<g, kCclThreads, 0, L.stream>>>(L.G, B.labels);
    cudaMemsetAsync(B.sizes, 0, sizeof(int) * (size_t)n, L.stream);
    k_ccl_flatten<<<g, kCclThreads, 0, L.stream>>>(n, B.labels, B.sizes);
    cudaMemsetAsync(B.count, 0, sizeof(int), L.stream);
    k_ccl_roots<<<g, kCclThreads, 0, L.stream>>>(n, B.labels, B.sizes, min_size, B.cap, B.count, B.pairs);
}

}  // namespace fre
