// Pipelined update kernels: the hot path of a time step for the shear and
// periodic devices with FP32 or 16-bit population storage.
//
// Persistent blocks walk over work units (a chunk of W consecutive x of one
// row (y, z), one node per thread).  Each block double-buffers its shared
// memory: while it computes unit k from one buffer, the 16-byte cp.async
// copies of unit k+1 (the pulled population rows and the phi/mu stencil
// rows, with 16-byte periodic halos in x) land in the other.  Results are
// written back into the buffer just read and leave with bulk asynchronous
// (TMA) stores, one per output row, so neither direction issues narrow
// per-thread requests.
#pragma once

#include <algorithm>

#include "fre_rows.cuh"

namespace fre {

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

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
__device__ __forceinline__ void mbar_init(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the mbarrier, for at most ~2 s; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
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

template <int Q, int FMT>
struct PipeLayout {
    using CL = ChunkLayout<Q, FMT>;
    static constexpr int NS = n_stencil_rows<Q>();
    __host__ __device__ static unsigned stage(int W) { return (CL::total(W, 2 * NS) + 127u) / 128u * 128u; }
    __host__ __device__ static unsigned smem(int W) { return 2 * stage(W); }
    // bytes the bulk copies of one unit deliver
    __host__ __device__ static unsigned tx_bytes(int W) { return CL::pop_bytes(W) + 2 * NS * CL::rw_f(W); }
};

// Stage the rows of unit `unit` into buffer `buf` with bulk copies that
// complete on the mbarrier `bar` (all threads take part).
template <int Q, int FMT, bool PULL>
__device__ __forceinline__ void stage_unit(const Launch &L, int W, int unit, unsigned char *buf, RowDesc *rows,
                                           unsigned *wall, unsigned bar) {
    using CL = ChunkLayout<Q, FMT>;
    constexpr int NS = n_stencil_rows<Q>();
    constexpr int NR = 2 * Q + 2 * NS;
    const Unit u = unit_at(L.G, W, unit);
    const unsigned foff = CL::field_off(W);
    if (threadIdx.x == 0) *wall = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < NR; k += blockDim.x) {
        if (k < 2 * Q) {
            const int lat = k >= Q, i = k - lat * Q;
            bool w;
            rows[k] = pop_row<Q, FMT>(L, L.src, lat, i, u.y, u.z, PULL, W, lat ? CL::g_off(W) : 0u, &w);
            if (w && !lat) atomicOr(wall, 1u << i);
        } else {
            const int j = k - 2 * Q, fld = j / NS, m = j - fld * NS;  // fld 0: phi, 1: mu
            const float *base = static_cast<const float *>(fld ? L.mu : L.phi);
            rows[k] = field_row<Q>(L, base, u.y, u.z, m, W, foff + fld * NS * CL::rw_f(W));
        }
    }
    __syncthreads();
    // one bulk copy per staged row when its halo-padded segment is contiguous
    // in global memory, else main part and wrapped halos separately
    if (threadIdx.x == 0) mbar_expect(bar, PipeLayout<Q, FMT>::tx_bytes(W));
    for (int k = threadIdx.x; k < NR; k += blockDim.x) {
        const RowDesc d = rows[k];
        const int H = 16 / (int)d.esz;
        const int nx = L.G.nx;
        unsigned char *dst = buf + d.dst;
        if (u.x0 >= H && u.x0 + W + H <= nx) {
            bulk_load(dst, d.src + (size_t)(u.x0 - H) * d.esz, (unsigned)((W + 2 * H) * d.esz), bar);
        } else {
            const int xl = u.x0 >= H ? u.x0 - H : nx - H;
            const int xr = (u.x0 + W < nx) ? u.x0 + W : 0;
            bulk_load(dst, d.src + (size_t)xl * d.esz, 16u, bar);
            bulk_load(dst + 16, d.src + (size_t)u.x0 * d.esz, (unsigned)(W * d.esz), bar);
            bulk_load(dst + 16 + W * d.esz, d.src + (size_t)xr * d.esz, 16u, bar);
        }
    }
}

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(256) k_update_pipe(Launch L, int W, int nunits) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    constexpr int NS = n_stencil_rows<Q>();
    constexpr int NR = 2 * Q + 2 * NS;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ RowDesc rows[NR];
    __shared__ unsigned wall_s[2];
    const unsigned stage_bytes = PipeLayout<Q, FMT>::stage(W);
    const unsigned foff = CL::field_off(W);
    const int xl = threadIdx.x;  // one node per thread, blockDim.x == W

    const float *php = static_cast<const float *>(L.phi_prev);
    const float rho0 = float(L.P.rho0);
    const float of = float(1.0 / L.P.tau_f), og = float(1.0 / L.P.tau_g);
    const float kf = float(1.0 - 0.5 / L.P.tau_f);
    const float g3 = float(3.0 * L.P.Gamma);
    const long long np = L.G.np;
    constexpr int c0 = stencil_slot<Q>(0, 0);

    __shared__ __align__(8) unsigned long long bars[2];
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bars[0]));
        mbar_init(smem_addr(&bars[1]));
        fence_async_smem();
    }
    __syncthreads();
    int unit = blockIdx.x;
    if (unit < nunits) stage_unit<Q, FMT, PULL>(L, W, unit, sm, rows, &wall_s[0], smem_addr(&bars[0]));
    for (int it = 0; unit < nunits; unit += gridDim.x, ++it) {
        const int b = it & 1;
        unsigned char *cur = sm + b * stage_bytes;
        unsigned char *nxt = sm + (b ^ 1) * stage_bytes;
        // the other buffer was the source of the previous unit's bulk stores
        bulk_wait_read();
        __syncthreads();
        const int next = unit + gridDim.x;
        if (next < nunits)
            stage_unit<Q, FMT, PULL>(L, W, next, nxt, rows, &wall_s[b ^ 1], smem_addr(&bars[b ^ 1]));
        if (!mbar_wait(smem_addr(&bars[b]), (unsigned)((it >> 1) & 1))) {
            if (threadIdx.x == 0) atomicExch(L.err, 1);
            return;
        }

        // ---- compute node xl of the current unit
        const Unit u = unit_at(L.G, W, unit);
        const unsigned wall = wall_s[b];
        const unsigned char *gb = cur + CL::g_off(W);
        const unsigned char *phs = cur + foff;
        const unsigned char *mus = cur + foff + NS * CL::rw_f(W);
        float f[Q], g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (PULL && (wall >> i) & 1u) {
                const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                const float cu = float(Lat<Q>::cx(i)) * uw;
                const float w2 = float(2.0 * Lat<Q>::w(i) * 3.0);
                // slot i holds the local row of population opp(i)
                const float fo = row_f_slot<Q, FMT>(cur, W, i, xl, float(Lat<Q>::w(Lat<Q>::opp(i))) * rho0);
                const float go = row_g<Q, FMT>(gb, W, i, xl);
                f[i] = fo + w2 * rho0 * cu;
                g[i] = go + w2 * php[u.row + u.x0 + xl] * cu;
            } else {
                const int xs = PULL ? xl - Lat<Q>::cx(i) : xl;
                f[i] = row_f<Q, FMT>(cur, W, i, xs, rho0);
                g[i] = row_g<Q, FMT>(gb, W, i, xs);
            }
        }
        float rho = 0.f, ph = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            ph += g[i];
            if (Lat<Q>::cx(i)) jx += float(Lat<Q>::cx(i)) * f[i];
            if (Lat<Q>::cy(i)) jy += float(Lat<Q>::cy(i)) * f[i];
            if (Lat<Q>::cz(i)) jz += float(Lat<Q>::cz(i)) * f[i];
        }
        float gpx = 0.f, gpy = 0.f, gpz = 0.f, gqx = 0.f, gqy = 0.f, gqz = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int slot = stencil_slot<Q>(Lat<Q>::cy(i), Lat<Q>::cz(i));
            const int xn = xl + Lat<Q>::cx(i);
            const float pv = row_field(phs, W, slot, xn);
            const float pm = pv * row_field(mus, W, slot, xn);
            const float w = float(Lat<Q>::w(i));
            if (Lat<Q>::cx(i)) { gpx += w * float(Lat<Q>::cx(i)) * pv; gqx += w * float(Lat<Q>::cx(i)) * pm; }
            if (Lat<Q>::cy(i)) { gpy += w * float(Lat<Q>::cy(i)) * pv; gqy += w * float(Lat<Q>::cy(i)) * pm; }
            if (Lat<Q>::cz(i)) { gpz += w * float(Lat<Q>::cz(i)) * pv; gqz += w * float(Lat<Q>::cz(i)) * pm; }
        }
        const float mu = row_field(mus, W, c0, xl);
        const float Fx = 3.f * (mu * gpx - gqx), Fy = 3.f * (mu * gpy - gqy), Fz = 3.f * (mu * gpz - gqz);
        const float inv = 1.f / rho;
        const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
        const float usq = ux * ux + uy * uy + uz * uz;
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const float gmu3 = g3 * mu;
        float fsum = 0.f, gsum = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float cx = float(Lat<Q>::cx(i)), cy = float(Lat<Q>::cy(i)), cz = float(Lat<Q>::cz(i));
            const float w = float(Lat<Q>::w(i));
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cF = cx * Fx + cy * Fy + cz * Fz;
            const float poly = 3.f * cu + 4.5f * cu * cu - 1.5f * usq;
            const float feq = w * rho * (1.f + poly);
            const float Sg = kf * w * (3.f * (cF - uF) + 9.f * cu * cF);
            const float fv = f[i] - (f[i] - feq) * of + Sg;
            const float geq = w * (gmu3 + ph * poly);
            const float gv = g[i] - (g[i] - geq) * og;
            fsum += fv;
            gsum += gv;
            f[i] = fv;
            g[i] = gv;
        }
        f[0] = rho - fsum;
        g[0] = ph - gsum;

        // ---- results into the buffer just read, then bulk stores
        __syncthreads();
        {
            S *fo = reinterpret_cast<S *>(cur);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (Fmt<FMT>::DEV) {
                    fo[i * W + xl] = from_float<S>(f[i] - float(Lat<Q>::w(i)) * rho0);
                    if (i > 0) fo[(Q + i - 1) * W + xl] = from_float<S>(g[i]);
                } else {
                    fo[i * W + xl] = f[i];
                    fo[(Q + i) * W + xl] = g[i];
                }
            }
            if constexpr (Fmt<FMT>::DEV) reinterpret_cast<float *>(fo + (2 * Q - 1) * W)[xl] = g[0];
        }
        fence_async_smem();
        __syncthreads();
        {
            // one output row per issuing thread: f rows, then g rows
            const size_t off = u.row + u.x0;
            const unsigned rb = (unsigned)(W * sizeof(S));
            bool issued = false;
            for (int k = threadIdx.x; k < 2 * Q; k += blockDim.x) {
                issued = true;
                if (k < Q) {
                    bulk_store(static_cast<S *>(L.dst.f) + (size_t)k * np + off, cur + k * rb, rb);
                } else if (!Fmt<FMT>::DEV) {
                    bulk_store(static_cast<S *>(L.dst.g) + (size_t)(k - Q) * np + off, cur + k * rb, rb);
                } else if (k == Q) {
                    bulk_store(L.dst.g0 + off, cur + (2 * Q - 1) * rb, (unsigned)(W * 4));
                } else {
                    bulk_store(static_cast<S *>(L.dst.g) + (size_t)(k - Q - 1) * np + off, cur + (k - 1) * rb, rb);
                }
            }
            if (issued) bulk_commit();
        }
    }
    bulk_wait_all();
}

// phi pass: pulled g rows -> phi, same pipeline; phi leaves with plain
// coalesced stores (4 bytes per node)
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(256) k_phi_pipe(Launch L, int W, int nunits) {
    using CL = ChunkLayout<Q, FMT>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ RowDesc rows[19];
    __shared__ unsigned wall_s[2];
    __shared__ __align__(8) unsigned long long bars[2];
    const unsigned stage_bytes = (CL::g_bytes(W) + 127u) / 128u * 128u;
    const int xl = threadIdx.x;
    const float *php = static_cast<const float *>(L.phi_prev);
    auto stage = [&](int unit, unsigned char *buf, unsigned *wall, unsigned bar) {
        const Unit u = unit_at(L.G, W, unit);
        if (threadIdx.x == 0) *wall = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < Q; k += blockDim.x) {
            bool w;
            rows[k] = pop_row<Q, FMT>(L, L.src, 1, k, u.y, u.z, PULL, W, 0u, &w);
            if (w) atomicOr(wall, 1u << k);
        }
        __syncthreads();
        if (threadIdx.x == 0) mbar_expect(bar, CL::g_bytes(W));
        for (int k = threadIdx.x; k < Q; k += blockDim.x) {
            const RowDesc d = rows[k];
            const int H = 16 / (int)d.esz;
            const int nx = L.G.nx;
            unsigned char *dst = buf + d.dst;
            if (u.x0 >= H && u.x0 + W + H <= nx) {
                bulk_load(dst, d.src + (size_t)(u.x0 - H) * d.esz, (unsigned)((W + 2 * H) * d.esz), bar);
            } else {
                const int xa = u.x0 >= H ? u.x0 - H : nx - H;
                const int xb = (u.x0 + W < nx) ? u.x0 + W : 0;
                bulk_load(dst, d.src + (size_t)xa * d.esz, 16u, bar);
                bulk_load(dst + 16, d.src + (size_t)u.x0 * d.esz, (unsigned)(W * d.esz), bar);
                bulk_load(dst + 16 + W * d.esz, d.src + (size_t)xb * d.esz, 16u, bar);
            }
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bars[0]));
        mbar_init(smem_addr(&bars[1]));
        fence_async_smem();
    }
    __syncthreads();
    int unit = blockIdx.x;
    if (unit < nunits) stage(unit, sm, &wall_s[0], smem_addr(&bars[0]));
    for (int it = 0; unit < nunits; unit += gridDim.x, ++it) {
        const int b = it & 1;
        unsigned char *cur = sm + b * stage_bytes;
        __syncthreads();  // the other buffer was read in the previous iteration
        const int next = unit + gridDim.x;
        if (next < nunits) stage(next, sm + (b ^ 1) * stage_bytes, &wall_s[b ^ 1], smem_addr(&bars[b ^ 1]));
        if (!mbar_wait(smem_addr(&bars[b]), (unsigned)((it >> 1) & 1))) {
            if (threadIdx.x == 0) atomicExch(L.err, 1);
            return;
        }
        const Unit u = unit_at(L.G, W, unit);
        const unsigned wall = wall_s[b];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (PULL && (wall >> i) & 1u) {
                const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                s += row_g<Q, FMT>(cur, W, i, xl) +
                     float(2.0 * Lat<Q>::w(i) * 3.0) * php[u.row + u.x0 + xl] * float(Lat<Q>::cx(i)) * uw;
            } else {
                s += row_g<Q, FMT>(cur, W, i, PULL ? xl - Lat<Q>::cx(i) : xl);
            }
        }
        static_cast<float *>(L.phi)[u.row + u.x0 + xl] = s;
    }
}

template <int Q, int FMT>
struct PipeLaunchers {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    static constexpr int kMaxSmem = 200 * 1024;
    static size_t smem_update(int W) { return PipeLayout<Q, FMT>::smem(W); }
    static size_t smem_phi(int W) { return 2 * ((CL::g_bytes(W) + 127u) / 128u * 128u); }

    // chunk width: one node per thread, W a multiple of 32 dividing nx
    static int width(const Geo &G, int pref) {
        if (G.device == FRE_FOUR_ROLLER) return 0;
        if ((G.np * sizeof(S)) % 16 != 0 || (G.nx * sizeof(S)) % 16 != 0) return 0;
        auto ok = [&](int W) {
            return W >= 32 && W <= 256 && W % 32 == 0 && G.nx % W == 0 && (W * sizeof(S)) % 16 == 0 &&
                   smem_update(W) <= (size_t)kMaxSmem;
        };
        if (pref > 0) return ok(pref) ? pref : 0;
        for (int W : {128, 64, 256, 32})
            if (ok(W)) return W;
        return 0;
    }
    // resident blocks per SM of a pipelined kernel (cached per kernel and W)
    static int blocks_per_sm(const void *fn, int W, size_t smem) {
        static const void *last_fn[16] = {};
        static int last_w[16] = {}, last_nb[16] = {};
        for (int k = 0; k < 16; ++k)
            if (last_fn[k] == fn && last_w[k] == W) return last_nb[k];
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, W, smem) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        if (nb < 1) nb = 1;
        static int slot = 0;
        last_fn[slot] = fn;
        last_w[slot] = W;
        last_nb[slot] = nb;
        slot = (slot + 1) & 15;
        return nb;
    }
    static bool configure() {
        static bool done = false;
        static bool ok = true;
        if (!done) {
            done = true;
            const int mx = kMaxSmem;
            ok &= cudaFuncSetAttribute(k_phi_pipe<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_phi_pipe<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_pipe<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_pipe<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_mu_rows<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
        }
        return ok;
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
    static int nunits(const Launch &L) { return (int)((size_t)L.G.ny * L.G.nz * (L.G.nx / L.W)); }
    static void phi(const Launch &L, bool pull) {
        const int nu = nunits(L);
        const size_t sm = smem_phi(L.W);
        if (pull) {
            const int g = std::min(nu, sms() * blocks_per_sm((const void *)k_phi_pipe<Q, FMT, true>, L.W, sm));
            k_phi_pipe<Q, FMT, true><<<g, L.W, sm, L.stream>>>(L, L.W, nu);
        } else {
            const int g = std::min(nu, sms() * blocks_per_sm((const void *)k_phi_pipe<Q, FMT, false>, L.W, sm));
            k_phi_pipe<Q, FMT, false><<<g, L.W, sm, L.stream>>>(L, L.W, nu);
        }
    }
    static void mu(const Launch &L) {
        k_mu_rows<Q><<<nunits(L), RowLaunchers<Q, FMT>::threads(L.W), RowLaunchers<Q, FMT>::smem_mu(L.W), L.stream>>>(
            L, L.W);
    }
    static void update(const Launch &L, bool pull) {
        const int nu = nunits(L);
        const size_t sm = smem_update(L.W);
        if (pull) {
            const int g = std::min(nu, sms() * blocks_per_sm((const void *)k_update_pipe<Q, FMT, true>, L.W, sm));
            k_update_pipe<Q, FMT, true><<<g, L.W, sm, L.stream>>>(L, L.W, nu);
        } else {
            const int g = std::min(nu, sms() * blocks_per_sm((const void *)k_update_pipe<Q, FMT, false>, L.W, sm));
            k_update_pipe<Q, FMT, false><<<g, L.W, sm, L.stream>>>(L, L.W, nu);
        }
    }
};

template <int Q, int FMT>
struct PipeEntry {
    static int width(const Geo &G, int pref) {
        const int W = PipeLaunchers<Q, FMT>::width(G, pref);
        return (W > 0 && PipeLaunchers<Q, FMT>::configure()) ? W : 0;
    }
};

// All kernels of one lattice and storage format.
template <int Q, int FMT>
const KernelSet *kernel_set_pipe() {
    using GL = Launchers<Q, FMT>;
    if constexpr (FMT == FRE_FP64) {
        return kernel_set<Q, FMT>();
    } else {
        using PL = PipeLaunchers<Q, FMT>;
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, PipeEntry<Q, FMT>::width, PL::phi,
                                     PL::mu, PL::update, nullptr, nullptr, nullptr, nullptr};
        return &ks;
    }
}

}  // namespace fre
