// Bulk asynchronous copies (TMA, cp.async.bulk) and mbarriers for the
// staged kernels, and the launch shape of persistent kernels.
#pragma once

#include <algorithm>
#include <mutex>

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
// dynamic shared-memory opt-in.  The tables are process-wide and shared by
// every context, so one mutex guards them (contexts may be created and
// stepped from several host threads at once); entries are per device.
struct LaunchShape {
    static std::mutex &lock() {
        static std::mutex m;
        return m;
    }
    static int device() {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            dev = 0;
        }
        return dev;
    }
    // raise a kernel's dynamic shared-memory opt-in to at least `smem`; one
    // record per kernel and device, so that no caller lowers what another
    // one raised (a launch above the opt-in fails with an invalid-argument
    // error)
    static void opt_in(const void *fn, size_t smem) {
        struct Rec {
            const void *fn;
            int dev;
            size_t smem;
        };
        static Rec recs[256] = {};
        static int n = 0;
        const int dev = device();
        std::lock_guard<std::mutex> g(lock());
        for (int k = 0; k < n; ++k) {
            if (recs[k].fn != fn || recs[k].dev != dev) continue;
            if (smem > recs[k].smem) {
                recs[k].smem = smem;
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            }
            return;
        }
        if (n < 256) recs[n++] = {fn, dev, smem};
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    // resident blocks per SM of a kernel (cached per kernel, device, block
    // size and shared memory)
    static int blocks_per_sm(const void *fn, int threads, size_t smem) {
        struct Rec {
            const void *fn;
            int dev, threads;
            size_t smem;
            int nb;
        };
        static Rec recs[32] = {};
        static int slot = 0;
        const int dev = device();
        std::lock_guard<std::mutex> g(lock());
        for (int k = 0; k < 32; ++k)
            if (recs[k].fn == fn && recs[k].dev == dev && recs[k].threads == threads && recs[k].smem == smem)
                return recs[k].nb;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        if (nb < 1) nb = 1;
        recs[slot] = {fn, dev, threads, smem, nb};
        slot = (slot + 1) & 31;
        return nb;
    }
    static int sms() {
        static int counts[64] = {};
        const int dev = device();
        std::lock_guard<std::mutex> g(lock());
        if (dev < 0 || dev >= 64) return 152;
        if (!counts[dev]) {
            int n = 0;
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            counts[dev] = n > 0 ? n : 1;
        }
        return counts[dev];
    }
};

}  // namespace fre
