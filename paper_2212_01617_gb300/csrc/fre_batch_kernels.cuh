// Batched per-node kernels: one launch advances every slot of a batch.  A
// persistent block walks a chunk of consecutive tiles, finds each tile's
// slot in the per-slot tile prefix, and runs the per-node code of the
// single-context kernels on that slot's launch descriptor (held in device
// memory, so the launch sequence can be captured in a CUDA graph).
#pragma once

#include <algorithm>

#include "fre_pipe.cuh"

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

// One launch over the tiles of every slot (tile = the BX x BY nodes of one
// z plane that a 256-thread block covers; block_start is the exclusive
// prefix of tiles per slot).  The grid is persistent: block b takes the
// `chunk` consecutive tiles from b * chunk, so that it crosses at most a few
// slot boundaries.  At each crossing warp 0 finds the slot and copies its
// launch descriptor into shared memory; every thread then reads the
// descriptor from there and the tile's corner follows from the tile's index
// within its slot.  The first descriptor is read before the wait for the
// previous kernel (the tables do not change during a step).  D2Q9 holds
// four blocks per SM (64 registers, 8 bytes of spill: 9.0 against 8.0 G node
// updates per second on the 64-case batch); D3Q19 would spill kilobytes.
template <int Q, int FMT, int BX, int KIND>
__global__ void __launch_bounds__(256, Q == 9 ? 4 : 1) k_batch(const Launch *__restrict__ cases, const int *__restrict__ start,
                                               int nslots, int ntiles, int chunk) {
    using T = typename Fmt<FMT>::T;
    constexpr int BY = 256 / BX;
    static_assert(sizeof(Launch) % 4 == 0, "descriptor copied in words");
    __shared__ Launch sL;
    __shared__ int s_begin, s_end;
    const int t0 = blockIdx.x * chunk;
    const int t1 = min(ntiles, t0 + chunk);
    bool waited = false;
    int begin = 0, end = 0;  // tiles of the current slot (the same in every thread)
    for (int tile = t0; tile < t1; ++tile) {
        if (tile >= end) {
            __syncthreads();  // the block is done with the previous descriptor
            if (threadIdx.x < 32) {
                const int slot = batch_slot(start, nslots, tile);
                const int *src = reinterpret_cast<const int *>(cases + slot);
                int *dst = reinterpret_cast<int *>(&sL);
                for (int k = threadIdx.x; k < (int)(sizeof(Launch) / 4); k += 32) dst[k] = __ldg(src + k);
                if (threadIdx.x == 0) {
                    s_begin = __ldg(start + slot);
                    s_end = __ldg(start + slot + 1);
                }
            }
            __syncthreads();
            begin = s_begin;
            end = s_end;
            if (!waited) {
                pdl_wait();
                waited = true;
            }
        }
        const Launch &L = sL;
        const int local = tile - begin;
        const int nbx = (L.G.nx + BX - 1) / BX, nby = (L.G.ny + BY - 1) / BY;
        const int tt = local / nbx;
        const int x = (local - tt * nbx) * BX + (int)(threadIdx.x % BX);
        const int y = (tt % nby) * BY + (int)(threadIdx.x / BX);
        const int z = tt / nby;
        if (x >= L.G.nx || y >= L.G.ny || z >= L.G.nz) continue;
        const Site s = make_site(L.G, x, y, z);
        if (is_solid(L.G, s.n)) continue;
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
}

// Ghost values at roller solids of every slot: tiles of 256 ghost nodes,
// persistent chunks as above (the descriptor read from global memory).
template <int Q, int FMT>
__global__ void __launch_bounds__(256) k_batch_ghost(const Launch *__restrict__ cases, const int *__restrict__ start,
                                                     int nslots, int field, int ntiles, int chunk) {
    using T = typename Fmt<FMT>::T;
    const int t0 = blockIdx.x * chunk;
    const int t1 = min(ntiles, t0 + chunk);
    pdl_wait();
    int slot = -1, end = 0;
    for (int tile = t0; tile < t1; ++tile) {
        if (tile >= end) {
            slot = batch_slot(start, nslots, tile);
            end = __ldg(start + slot + 1);
        }
        const Launch &L = cases[slot];
        const int t = (tile - __ldg(start + slot)) * 256 + threadIdx.x;
        if (t < L.n_ghost) node_ghost<Q, T>(L, static_cast<T *>(field ? L.mu : L.phi), t);
    }
}

// persistent grid of a tile loop: as many blocks as fit on the GPU at once,
// each with an equal chunk of consecutive tiles
inline void tile_chunks(const void *fn, int ntiles, int &grid, int &chunk) {
    const int cap = std::max(1, LaunchShape::sms() * LaunchShape::blocks_per_sm(fn, 256, 0));
    chunk = (ntiles + cap - 1) / cap;
    grid = (ntiles + chunk - 1) / chunk;
}

template <int Q, int FMT>
struct BatchLaunchers {
    template <int KIND, int BX>
    static void go(const BatchLaunch &B) {
        auto fn = k_batch<Q, FMT, BX, KIND>;
        int grid, chunk;
        tile_chunks((const void *)fn, B.total_blocks, grid, chunk);
        launch_pdl(fn, dim3(grid), dim3(256), 0, B.stream, B.cases, B.block_start, B.nslots, B.total_blocks, chunk);
    }
    template <int KIND>
    static void run(const BatchLaunch &B, int bx) {
        if (B.total_blocks <= 0) return;
        switch (bx) {
            case 32: go<KIND, 32>(B); break;
            case 128: go<KIND, 128>(B); break;
            default: go<KIND, 64>(B); break;
        }
    }
    static void phi(const BatchLaunch &B, int bx) { run<B_PHI>(B, bx); }
    static void mu(const BatchLaunch &B, int bx) { run<B_MU>(B, bx); }
    static void update(const BatchLaunch &B, int bx) { run<B_UPDATE>(B, bx); }
    static void ghost(const BatchLaunch &B, int field) {
        if (B.total_ghost_blocks <= 0) return;
        auto fn = k_batch_ghost<Q, FMT>;
        int grid, chunk;
        tile_chunks((const void *)fn, B.total_ghost_blocks, grid, chunk);
        launch_pdl(fn, dim3(grid), dim3(256), 0, B.stream, B.cases, B.ghost_start, B.nslots, field,
                   B.total_ghost_blocks, chunk);
    }
    static const BatchKernels *set() {
        static const BatchKernels k = {phi, mu, ghost, update};
        return &k;
    }
};

}  // namespace fre
