// Batched per-node kernels: one launch advances every slot of a batch.  A
// block finds its slot by binary search in the per-slot block prefix, then
// runs the per-node code of the single-context kernels on that slot's
// launch descriptor (held in device memory, so the launch sequence can be
// captured in a CUDA graph).
#pragma once

#include "fre_kernels.cuh"

namespace fre {

__device__ __forceinline__ int batch_slot(const int *start, int nslots, int b) {
    int lo = 0, hi = nslots;  // start[lo] <= b < start[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

enum BatchKind { B_PHI = 0, B_MU = 1, B_UPDATE = 2 };

template <int Q, int FMT, int BX, int KIND>
__global__ void __launch_bounds__(256) k_batch(const Launch *__restrict__ cases, const int *__restrict__ start,
                                               int nslots) {
    using T = typename Fmt<FMT>::T;
    constexpr int BY = 256 / BX;
    static_assert(sizeof(Launch) % 4 == 0, "descriptor copied in words");
    // The block's slot, its launch descriptor and the block's corner in that
    // lattice are found once per block by the first warp and shared: every
    // thread then reads the descriptor from shared memory and does no
    // division of its own.
    __shared__ Launch sL;
    __shared__ int corner[3];
    if (threadIdx.x < 32) {
        const int slot = batch_slot(start, nslots, blockIdx.x);
        const int *src = reinterpret_cast<const int *>(cases + slot);
        int *dst = reinterpret_cast<int *>(&sL);
        for (int k = threadIdx.x; k < (int)(sizeof(Launch) / 4); k += 32) dst[k] = __ldg(src + k);
        if (threadIdx.x == 0) {
            const int nx = __ldg(&cases[slot].G.nx), ny = __ldg(&cases[slot].G.ny);
            const int local = blockIdx.x - __ldg(start + slot);
            const int nbx = (nx + BX - 1) / BX, nby = (ny + BY - 1) / BY;
            const int t = local / nbx;
            corner[0] = (local - t * nbx) * BX;
            corner[1] = (t % nby) * BY;
            corner[2] = t / nby;
        }
    }
    __syncthreads();
    pdl_wait();
    const Launch &L = sL;
    const int x = corner[0] + (int)(threadIdx.x % BX), y = corner[1] + (int)(threadIdx.x / BX), z = corner[2];
    if (x >= L.G.nx || y >= L.G.ny || z >= L.G.nz) return;
    const Site s = make_site(L.G, x, y, z);
    if (is_solid(L.G, s.n)) return;
    if (KIND == B_MU) {
        node_mu<Q, T>(L, s);
    } else if (KIND == B_PHI) {
        if (L.pull) node_phi<Q, FMT, true>(L, s);
        else node_phi<Q, FMT, false>(L, s);
    } else {
        if (L.pull) node_update<Q, FMT, true>(L, s);
        else node_update<Q, FMT, false>(L, s);
    }
}

template <int Q, int FMT>
__global__ void __launch_bounds__(256) k_batch_ghost(const Launch *__restrict__ cases, const int *__restrict__ start,
                                                     int nslots, int field) {
    using T = typename Fmt<FMT>::T;
    const int slot = batch_slot(start, nslots, blockIdx.x);
    const Launch &L = cases[slot];
    const int t = (blockIdx.x - __ldg(start + slot)) * 256 + threadIdx.x;
    pdl_wait();
    if (t >= L.n_ghost) return;
    node_ghost<Q, T>(L, static_cast<T *>(field ? L.mu : L.phi), t);
}

template <int Q, int FMT>
struct BatchLaunchers {
    template <int KIND>
    static void run(const BatchLaunch &B, int bx) {
        if (B.total_blocks <= 0) return;
        switch (bx) {
            case 32: launch_pdl(k_batch<Q, FMT, 32, KIND>, dim3(B.total_blocks), dim3(256), 0, B.stream, B.cases, B.block_start, B.nslots); break;
            case 128: launch_pdl(k_batch<Q, FMT, 128, KIND>, dim3(B.total_blocks), dim3(256), 0, B.stream, B.cases, B.block_start, B.nslots); break;
            default: launch_pdl(k_batch<Q, FMT, 64, KIND>, dim3(B.total_blocks), dim3(256), 0, B.stream, B.cases, B.block_start, B.nslots); break;
        }
    }
    static void phi(const BatchLaunch &B, int bx) { run<B_PHI>(B, bx); }
    static void mu(const BatchLaunch &B, int bx) { run<B_MU>(B, bx); }
    static void update(const BatchLaunch &B, int bx) { run<B_UPDATE>(B, bx); }
    static void ghost(const BatchLaunch &B, int field) {
        if (B.total_ghost_blocks > 0)
            launch_pdl(k_batch_ghost<Q, FMT>, dim3(B.total_ghost_blocks), dim3(256), 0, B.stream, B.cases, B.ghost_start, B.nslots, field);
    }
    static const BatchKernels *set() {
        static const BatchKernels k = {phi, mu, ghost, update};
        return &k;
    }
};

}  // namespace fre
