// Bulk asynchronous copies (TMA, cp.async.bulk) and mbarriers for the
// staged kernels, and the launch shape of persistent kernels.
#pragma once

#include <algorithm>

#include "fre_rows.cuh"

namespace fre {

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bulk (TMA) store of `bytes` (multiple of 16) from shared to global memory
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the shared-memory sources of all committed bulk stores are read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until all committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// bulk (TMA) load of `bytes` (multiple of 16) from global to shared memory,
// completing on the mbarrier `bar`
__device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ Unit unit_at(const Geo &G, int W, int b) {
    const int nch = G.nx / W;
    const int r = b / nch;
    Unit u;
    u.x0 = (b - r * nch) * W;
    u.y = r % G.ny;
    u.z = r / G.ny;
    u.row = (size_t)r * G.nx;
    return u;
}

// Launch shape of the persistent kernels: SM count, resident blocks and the
// dynamic shared-memory opt-in.
struct LaunchShape {
    // raise a kernel's dynamic shared-memory opt-in to at least `smem`; one
    // record per kernel, so that no caller lowers what another one raised
    // (a launch above the opt-in fails with an invalid-argument error)
    static void opt_in(const void *fn, size_t smem) {
        static const void *fns[128] = {};
        static size_t vals[128] = {};
        static int n = 0;
        for (int k = 0; k < n; ++k) {
            if (fns[k] != fn) continue;
            if (smem > vals[k]) {
                vals[k] = smem;
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            }
            return;
        }
        if (n < 128) {
            fns[n] = fn;
            vals[n] = smem;
            ++n;
        }
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    // resident blocks per SM of a kernel (cached per kernel and block size)
    static int blocks_per_sm(const void *fn, int threads, size_t smem) {
        static const void *last_fn[16] = {};
        static int last_t[16] = {}, last_nb[16] = {};
        for (int k = 0; k < 16; ++k)
            if (last_fn[k] == fn && last_t[k] == threads) return last_nb[k];
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        if (nb < 1) nb = 1;
        static int slot = 0;
        last_fn[slot] = fn;
        last_t[slot] = threads;
        last_nb[slot] = nb;
        slot = (slot + 1) & 15;
        return nb;
    }
    static int sms() {
        static int n = 0;
        if (!n) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (n <= 0) n = 1;
        }
        return n;
    }
};

}  // namespace fre
