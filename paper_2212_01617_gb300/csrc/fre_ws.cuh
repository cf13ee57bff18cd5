// Warp-specialised pipelined kernels: the hot path of a time step for the
// shear and periodic devices with FP32 or 16-bit population storage.
//
// A persistent block = one producer warp + W/32 consumer warps.  Work unit:
// a chunk of W consecutive x of one row (y, z), one node per consumer
// thread.  The producer walks the block's units, builds the table of rows a
// unit needs (pulled population rows shifted by -c_i in y and z, phi/mu
// stencil rows) and stages them into an NST-deep ring of shared-memory
// buffers with bulk (TMA) copies that complete on the stage's `full`
// mbarrier.  Consumers wait on `full`, compute, write their results back
// into the stage, and one consumer thread sends them out with bulk (TMA)
// stores, waits until those have read the stage and arrives on `empty`,
// which hands the stage back to the producer.  Every mbarrier wait is
// bounded in time; on timeout the block records an error code and leaves
// through a path every thread of a role takes together.
#pragma once

#include "fre_pipe.cuh"

namespace fre {

__device__ __forceinline__ void mbar_init_count(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait with a suspend hint (the warp sleeps in hardware instead of
// spinning); false after ~2 s.
__device__ __forceinline__ bool mbar_wait_hint(unsigned bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(1000000u)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}
// named barrier among the consumer threads only (id 1)
__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Issue the bulk loads of one staged row for chunk [x0, x0 + W).
__device__ __forceinline__ void load_row(const RowDesc &d, unsigned char *buf, int x0, int W, int nx,
                                         unsigned bar) {
    const int H = 16 / (int)d.esz;
    unsigned char *dst = buf + d.dst;
    if (x0 >= H && x0 + W + H <= nx) {
        bulk_load(dst, d.src + (size_t)(x0 - H) * d.esz, (unsigned)((W + 2 * H) * d.esz), bar);
    } else {
        const int xa = x0 >= H ? x0 - H : nx - H;
        const int xb = (x0 + W < nx) ? x0 + W : 0;
        bulk_load(dst, d.src + (size_t)xa * d.esz, 16u, bar);
        bulk_load(dst + 16, d.src + (size_t)x0 * d.esz, (unsigned)(W * d.esz), bar);
        bulk_load(dst + 16 + W * d.esz, d.src + (size_t)xb * d.esz, 16u, bar);
    }
}

enum WsKind { WS_UPDATE = 0, WS_PHI = 1, WS_MU = 2 };

// Rows a unit stages, per kernel kind.
template <int Q, int FMT, int KIND>
struct WsRows {
    using CL = ChunkLayout<Q, FMT>;
    static constexpr int NS = n_stencil_rows<Q>();
    static constexpr int NR = KIND == WS_UPDATE ? 2 * Q + 2 * NS : (KIND == WS_PHI ? Q : NS);
    __host__ __device__ static unsigned tx_bytes(int W) {
        if (KIND == WS_UPDATE) return CL::pop_bytes(W) + 2 * NS * CL::rw_f(W);
        if (KIND == WS_PHI) return CL::g_bytes(W);
        return NS * CL::rw_f(W);
    }
    __host__ __device__ static unsigned stage_bytes(int W) {
        unsigned b = KIND == WS_UPDATE ? CL::total(W, 2 * NS) : tx_bytes(W);
        return (b + 127u) / 128u * 128u;
    }
    // row k of the unit; *wall set for a population wall link of f (update)
    // or g (phi)
    template <bool PULL>
    __device__ static RowDesc row(const Launch &L, const Unit &u, int W, int k, bool *wall) {
        *wall = false;
        if (KIND == WS_UPDATE) {
            if (k < 2 * Q) {
                const int lat = k >= Q, i = k - lat * Q;
                bool w;
                RowDesc d = pop_row<Q, FMT>(L, L.src, lat, i, u.y, u.z, PULL, W, lat ? CL::g_off(W) : 0u, &w);
                *wall = w && !lat;
                return d;
            }
            const int j = k - 2 * Q, fld = j / NS, m = j - fld * NS;
            const float *base = static_cast<const float *>(fld ? L.mu : L.phi);
            return field_row<Q>(L, base, u.y, u.z, m, W, CL::field_off(W) + fld * NS * CL::rw_f(W));
        } else if (KIND == WS_PHI) {
            bool w;
            RowDesc d = pop_row<Q, FMT>(L, L.src, 1, k, u.y, u.z, PULL, W, 0u, &w);
            *wall = w;
            return d;
        } else {
            return field_row<Q>(L, static_cast<const float *>(L.phi), u.y, u.z, k, W, 0u);
        }
    }
};

template <int Q, int FMT, int KIND, bool PULL, int NST>
__global__ void __launch_bounds__(288) k_ws(Launch L, int W, int nunits) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    using R = WsRows<Q, FMT, KIND>;
    constexpr int NS = n_stencil_rows<Q>();
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) unsigned long long full[NST], empty[NST];
    __shared__ unsigned wall_s[NST];
    // set by consumers only, before a consumer barrier, read after it: every
    // consumer leaves the loop at the same unit
    __shared__ int cabort;
    const int ncons = W;  // consumer threads
    const bool producer = threadIdx.x >= ncons;
    const unsigned stage_bytes = R::stage_bytes(W);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init_count(smem_addr(&full[s]), 1);
            mbar_init_count(smem_addr(&empty[s]), 1);
        }
        cabort = 0;
        fence_async_smem();
    }
    __syncthreads();

    if (producer) {
        // ------------------------------------------------------ producer warp
        const int lane = threadIdx.x - ncons;
        int k = 0;
        for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
            const int s = k % NST;
            if (k >= NST) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_hint(smem_addr(&empty[s]), (unsigned)(((k / NST) - 1) & 1));
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    if (lane == 0) atomicExch(L.err, 2);
                    break;  // consumers then time out on `full` and leave together
                }
            }
            const Unit u = unit_at(L.G, W, unit);
            unsigned char *buf = sm + s * stage_bytes;
            const unsigned bar = smem_addr(&full[s]);
            RowDesc d0, d1;
            bool w0 = false, w1 = false;
            const bool has0 = lane < R::NR, has1 = lane + 32 < R::NR;
            if (has0) d0 = R::template row<PULL>(L, u, W, lane, &w0);
            if (has1) d1 = R::template row<PULL>(L, u, W, lane + 32, &w1);
            (void)w1;  // rows 32.. are never population rows with wall links (q <= 19)
            const unsigned wall = __ballot_sync(0xffffffffu, w0 && lane < Q);
            if (lane == 0) {
                wall_s[s] = wall;
                mbar_expect(bar, R::tx_bytes(W));
            }
            __syncwarp();
            if (has0) load_row(d0, buf, u.x0, W, L.G.nx, bar);
            if (has1) load_row(d1, buf, u.x0, W, L.G.nx, bar);
        }
        return;
    }

    // ------------------------------------------------------------ consumers
    const int xl = threadIdx.x;
    const float *php = static_cast<const float *>(L.phi_prev);
    const float rho0 = float(L.P.rho0);
    int k = 0;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
        const int s = k % NST;
        unsigned char *cur = sm + s * stage_bytes;
        const bool ok = mbar_wait_hint(smem_addr(&full[s]), (unsigned)((k / NST) & 1));
        if (!ok) {
            atomicExch(L.err, 3);
            cabort = 1;
        }
        consumer_sync(ncons);
        if (cabort) break;
        const Unit u = unit_at(L.G, W, unit);
        const unsigned wall = wall_s[s];

        if constexpr (KIND == WS_PHI) {
            float sum = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                    sum += row_g<Q, FMT>(cur, W, i, xl) +
                           float(2.0 * Lat<Q>::w(i) * 3.0) * php[u.row + u.x0 + xl] * float(Lat<Q>::cx(i)) * uw;
                } else {
                    sum += row_g<Q, FMT>(cur, W, i, PULL ? xl - Lat<Q>::cx(i) : xl);
                }
            }
            consumer_sync(ncons);  // every consumer has read the stage
            if (xl == 0) mbar_arrive(smem_addr(&empty[s]));
            static_cast<float *>(L.phi)[u.row + u.x0 + xl] = sum;
        } else if constexpr (KIND == WS_MU) {
            constexpr int c0 = stencil_slot<Q>(0, 0);
            const float p0 = row_field(cur, W, c0, xl);
            float lap = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int slot = stencil_slot<Q>(Lat<Q>::cy(i), Lat<Q>::cz(i));
                lap += float(Lat<Q>::w(i)) * (row_field(cur, W, slot, xl + Lat<Q>::cx(i)) - p0);
            }
            lap *= 6.f;
            consumer_sync(ncons);
            if (xl == 0) mbar_arrive(smem_addr(&empty[s]));
            static_cast<float *>(L.mu)[u.row + u.x0 + xl] =
                float(L.P.A) * (p0 * p0 * p0 - p0) - float(L.P.kappa) * lap;
        } else {
            const unsigned foff = CL::field_off(W);
            const unsigned char *gb = cur + CL::g_off(W);
            const unsigned char *phs = cur + foff;
            const unsigned char *mus = cur + foff + NS * CL::rw_f(W);
            const float of = float(1.0 / L.P.tau_f), og = float(1.0 / L.P.tau_g);
            const float kf = float(1.0 - 0.5 / L.P.tau_f);
            const float g3 = float(3.0 * L.P.Gamma);
            constexpr int c0 = stencil_slot<Q>(0, 0);
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

            // results into the stage just read, then bulk stores
            consumer_sync(ncons);
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
            fence_async_smem();
            consumer_sync(ncons);
            if (xl < 32) {
                // warp 0 sends the unit's output rows; lane j takes rows j, j + 32
                const size_t off = u.row + u.x0;
                const unsigned rb = (unsigned)(W * sizeof(S));
                const long long np = L.G.np;
                for (int r = xl; r < 2 * Q; r += 32) {
                    if (r < Q) {
                        bulk_store(static_cast<S *>(L.dst.f) + (size_t)r * np + off, cur + r * rb, rb);
                    } else if (!Fmt<FMT>::DEV) {
                        bulk_store(static_cast<S *>(L.dst.g) + (size_t)(r - Q) * np + off, cur + r * rb, rb);
                    } else if (r == Q) {
                        bulk_store(L.dst.g0 + off, cur + (2 * Q - 1) * rb, (unsigned)(W * 4));
                    } else {
                        bulk_store(static_cast<S *>(L.dst.g) + (size_t)(r - Q - 1) * np + off, cur + (r - 1) * rb,
                                   rb);
                    }
                }
                bulk_commit();
                bulk_wait_read();
                __syncwarp();
                if (xl == 0) mbar_arrive(smem_addr(&empty[s]));
            }
        }
    }
    if (KIND == WS_UPDATE && xl < 32) bulk_wait_all();
}

template <int Q, int FMT>
struct WsLaunchers {
    using S = typename Fmt<FMT>::S;
    static constexpr int kMaxSmem = 200 * 1024;
    template <int KIND>
    static int nst(int W) {
        const unsigned sb = WsRows<Q, FMT, KIND>::stage_bytes(W);
        return 3 * sb <= (unsigned)kMaxSmem ? 3 : 2;
    }
    // chunk width: consumer threads = W (one node each), a multiple of 32
    static int width(const Geo &G, int pref) {
        if (G.device == FRE_FOUR_ROLLER) return 0;
        if ((G.np * sizeof(S)) % 16 != 0 || (G.nx * sizeof(S)) % 16 != 0) return 0;
        auto ok = [&](int W) {
            return W >= 32 && W <= 256 && W % 32 == 0 && G.nx % W == 0 && (W * sizeof(S)) % 16 == 0 &&
                   2 * WsRows<Q, FMT, WS_UPDATE>::stage_bytes(W) <= (unsigned)kMaxSmem;
        };
        if (pref > 0) return ok(pref) ? pref : 0;
        for (int W : {128, 256, 64, 32})
            if (ok(W)) return W;
        return 0;
    }
    template <int KIND, bool PULL, int NST>
    static void launch(const Launch &L) {
        const int W = L.W;
        const int nu = (int)((size_t)L.G.ny * L.G.nz * (L.G.nx / W));
        const size_t smem = (size_t)NST * WsRows<Q, FMT, KIND>::stage_bytes(W);
        auto fn = k_ws<Q, FMT, KIND, PULL, NST>;
        static bool attr = false;
        if (!attr) {
            attr = true;
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        }
        const int g = std::min(nu, PipeLaunchers<Q, FMT>::sms() *
                                       PipeLaunchers<Q, FMT>::blocks_per_sm((const void *)fn, W + 32, smem));
        fn<<<g, W + 32, smem, L.stream>>>(L, W, nu);
    }
    template <int KIND, bool PULL>
    static void run(const Launch &L) {
        if (nst<KIND>(L.W) == 3) launch<KIND, PULL, 3>(L);
        else launch<KIND, PULL, 2>(L);
    }
    static void phi(const Launch &L, bool pull) {
        if (pull) run<WS_PHI, true>(L);
        else run<WS_PHI, false>(L);
    }
    static void mu(const Launch &L) { run<WS_MU, true>(L); }
    static void update(const Launch &L, bool pull) {
        if (pull) run<WS_UPDATE, true>(L);
        else run<WS_UPDATE, false>(L);
    }
};

template <int Q, int FMT>
struct WsEntry {
    static int width(const Geo &G, int pref) { return WsLaunchers<Q, FMT>::width(G, pref); }
};

}  // namespace fre

namespace fre {

// -------------------------------------------------------------------------
// Full-row variants: one work unit = one whole x-row (y, z), so every staged
// row is a single large bulk copy (nx * element bytes) -- few, large TMA
// operations keep HBM busy where many small ones do not.  The periodic x
// shift is a modular index into the staged row.  Consumer thread t updates
// the adjacent nodes x = 2t, 2t + 1 and stores 2-wide vectors.
//   KIND WS_PHI   : stages the q pulled g rows, writes phi
//   KIND WS_MU    : stages the phi rows of the stencil, writes mu
//   KIND WS_UPDATE: stages the 2q pulled f and g rows; the phi/mu stencil
//                   values come from global memory (re-read by the nine
//                   neighbouring rows, they stay in L2)

// Axial stencil slots (cy, cz) with cy == 0 or cz == 0: the only ones whose
// directions carry an x shift.  D3Q19: (0,0) (1,0) (-1,0) (0,1) (0,-1);
// D2Q9: (0,0) (1,0) (-1,0).
template <int Q>
__host__ __device__ constexpr int n_axial() { return Lat<Q>::D == 2 ? 3 : 5; }
__host__ __device__ constexpr int axial_slot(int cy, int cz) {
    return (cy == 0 && cz == 0) ? 0 : (cz == 0 ? (cy > 0 ? 1 : 2) : (cy == 0 ? (cz > 0 ? 3 : 4) : -1));
}
__host__ __device__ constexpr int axial_cy(int a) { return a == 1 ? 1 : (a == 2 ? -1 : 0); }
__host__ __device__ constexpr int axial_cz(int a) { return a == 3 ? 1 : (a == 4 ? -1 : 0); }

template <int Q, int FMT, int KIND>
struct FullRowLayout {
    using S = typename Fmt<FMT>::S;
    static constexpr bool DEV = Fmt<FMT>::DEV;
    static constexpr int NS = n_stencil_rows<Q>();
    static constexpr int NA = n_axial<Q>();
    __host__ __device__ static unsigned rowb(int nx) { return (unsigned)(nx * sizeof(S)); }
    // start of the g rows
    __host__ __device__ static unsigned g_off(int nx) { return KIND == WS_UPDATE ? Q * rowb(nx) : 0u; }
    __host__ __device__ static unsigned g_bytes(int nx) {
        return DEV ? (Q - 1) * rowb(nx) + (unsigned)nx * 4 : Q * rowb(nx);
    }
    // update: axial phi rows then axial mu rows after the populations
    __host__ __device__ static unsigned f_off(int nx) { return (g_off(nx) + g_bytes(nx) + 15u) / 16u * 16u; }
    __host__ __device__ static unsigned bytes(int nx) {
        if (KIND == WS_MU) return NS * (unsigned)nx * 4;
        if (KIND == WS_UPDATE) return f_off(nx) + 2 * NA * (unsigned)nx * 4;
        return g_off(nx) + g_bytes(nx);
    }
    __host__ __device__ static unsigned stage(int nx) { return (bytes(nx) + 127u) / 128u * 128u; }
    __host__ __device__ static int nrows() {
        return KIND == WS_UPDATE ? 2 * Q + 2 * NA : (KIND == WS_PHI ? Q : NS);
    }
};

__device__ __forceinline__ int wrap_x(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

template <int Q, int FMT>
__device__ __forceinline__ float fr_g(const unsigned char *gb, int nx, int i, int xs) {
    using S = typename Fmt<FMT>::S;
    if constexpr (Fmt<FMT>::DEV) {
        if (i == 0) return reinterpret_cast<const float *>(gb + (size_t)(Q - 1) * nx * sizeof(S))[xs];
        return to_float(reinterpret_cast<const S *>(gb)[(size_t)(i - 1) * nx + xs]);
    } else {
        return reinterpret_cast<const S *>(gb)[(size_t)i * nx + xs];
    }
}

template <int Q, int FMT, int KIND, bool PULL, int NST, int NPT>
__global__ void __launch_bounds__(544, 1) k_wsrow(Launch L, int nunits) {
    using S = typename Fmt<FMT>::S;
    using FL = FullRowLayout<Q, FMT, KIND>;
    constexpr int NS = n_stencil_rows<Q>();
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) unsigned long long full[NST], empty[NST];
    __shared__ unsigned wall_s[NST];
    __shared__ int cabort;
    const int nx = L.G.nx;
    const int ncons = nx / NPT;
    const bool producer = threadIdx.x >= ncons;
    const unsigned stage_bytes = FL::stage(nx);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init_count(smem_addr(&full[s]), 1);
            mbar_init_count(smem_addr(&empty[s]), 1);
        }
        cabort = 0;
        fence_async_smem();
    }
    __syncthreads();

    if (producer) {
        const int lane = threadIdx.x - ncons;
        int k = 0;
        for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
            const int s = k % NST;
            if (k >= NST) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_hint(smem_addr(&empty[s]), (unsigned)(((k / NST) - 1) & 1));
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    if (lane == 0) atomicExch(L.err, 4);
                    break;  // consumers then time out on `full` and leave together
                }
            }
            const int y = unit % L.G.ny, z = unit / L.G.ny;
            unsigned char *buf = sm + s * stage_bytes;
            const unsigned bar = smem_addr(&full[s]);
            unsigned wall = 0;
            const char *src[2];
            unsigned dst[2], nb[2];
            int cnt = 0;
            for (int r = lane; r < FL::nrows(); r += 32, ++cnt) {
                if (KIND == WS_UPDATE && r >= 2 * Q) {
                    const int j = r - 2 * Q, fld = j / FL::NA, a = j - fld * FL::NA;
                    int yn = y + axial_cy(a);
                    yn = (L.G.device == FRE_SHEAR) ? (yn < 0 ? 0 : (yn >= L.G.ny ? L.G.ny - 1 : yn))
                                                   : wrapi(yn, L.G.ny);
                    const int zn = wrapi(z + axial_cz(a), L.G.nz);
                    const float *base = static_cast<const float *>(fld ? L.mu : L.phi);
                    src[cnt] = reinterpret_cast<const char *>(base + ((size_t)zn * L.G.ny + yn) * nx);
                    dst[cnt] = FL::f_off(nx) + (unsigned)(j * nx * 4);
                    nb[cnt] = (unsigned)(nx * 4);
                    continue;
                }
                if (KIND == WS_MU) {
                    const int cy = (Lat<Q>::D == 2 ? r : r % 3) - 1, cz = Lat<Q>::D == 2 ? 0 : r / 3 - 1;
                    int yn = y + cy;
                    yn = (L.G.device == FRE_SHEAR) ? (yn < 0 ? 0 : (yn >= L.G.ny ? L.G.ny - 1 : yn))
                                                   : wrapi(yn, L.G.ny);
                    const int zn = wrapi(z + cz, L.G.nz);
                    src[cnt] = reinterpret_cast<const char *>(static_cast<const float *>(L.phi) +
                                                              ((size_t)zn * L.G.ny + yn) * nx);
                    dst[cnt] = (unsigned)(r * nx * 4);
                    nb[cnt] = (unsigned)(nx * 4);
                    continue;
                }
                const int lat = (KIND == WS_PHI) ? 1 : (r >= Q);
                const int i = (KIND == WS_PHI) ? r : r - lat * Q;
                int ys, zs, pi = i;
                if (!src_row<Q>(L.G, y, z, i, PULL, ys, zs)) {
                    wall |= 1u << i;
                    ys = y;
                    zs = z;
                    pi = Lat<Q>::opp(i);
                }
                const size_t row = ((size_t)zs * L.G.ny + ys) * nx;
                if (!lat) {
                    src[cnt] = static_cast<const char *>(L.src.f) + ((size_t)pi * L.G.np + row) * sizeof(S);
                    dst[cnt] = i * FL::rowb(nx);
                    nb[cnt] = FL::rowb(nx);
                } else if (!Fmt<FMT>::DEV) {
                    src[cnt] = static_cast<const char *>(L.src.g) + ((size_t)pi * L.G.np + row) * sizeof(S);
                    dst[cnt] = FL::g_off(nx) + i * FL::rowb(nx);
                    nb[cnt] = FL::rowb(nx);
                } else if (pi == 0) {  // only for i = 0 (opp(i) = 0 iff i = 0)
                    src[cnt] = reinterpret_cast<const char *>(L.src.g0 + row);
                    dst[cnt] = FL::g_off(nx) + (Q - 1) * FL::rowb(nx);
                    nb[cnt] = (unsigned)(nx * 4);
                } else {
                    src[cnt] = static_cast<const char *>(L.src.g) + ((size_t)(pi - 1) * L.G.np + row) * sizeof(S);
                    dst[cnt] = FL::g_off(nx) + (i - 1) * FL::rowb(nx);
                    nb[cnt] = FL::rowb(nx);
                }
            }
            wall = __reduce_or_sync(0xffffffffu, wall);
            if (lane == 0) {
                wall_s[s] = wall;
                mbar_expect(bar, FL::bytes(nx));
            }
            __syncwarp();
            for (int c = 0; c < cnt; ++c) bulk_load(buf + dst[c], src[c], nb[c], bar);
        }
        return;
    }

    // ------------------------------------------------------------ consumers
    const float rho0 = float(L.P.rho0);
    const float *__restrict__ php = static_cast<const float *>(L.phi_prev);
    const long long np = L.G.np;
    int k = 0;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
        const int s = k % NST;
        const unsigned char *cur = sm + s * stage_bytes;
        const unsigned char *gb = cur + FL::g_off(nx);
        const bool ok = mbar_wait_hint(smem_addr(&full[s]), (unsigned)((k / NST) & 1));
        if (!ok) {
            atomicExch(L.err, 5);
            cabort = 1;
        }
        consumer_sync(ncons);
        if (cabort) break;
        const int y = unit % L.G.ny, z = unit / L.G.ny;
        const unsigned wall = wall_s[s];
        const size_t row = ((size_t)z * L.G.ny + y) * nx;
        const int x0 = 2 * threadIdx.x;

        if constexpr (KIND == WS_PHI) {
            float out[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int x = x0 + t;
                float sum = 0.f;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (PULL && (wall >> i) & 1u) {
                        const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                        sum += fr_g<Q, FMT>(gb, nx, i, x) +
                               float(2.0 * Lat<Q>::w(i) * 3.0) * php[row + x] * float(Lat<Q>::cx(i)) * uw;
                    } else {
                        sum += fr_g<Q, FMT>(gb, nx, i, PULL ? wrap_x(x - Lat<Q>::cx(i), nx) : x);
                    }
                }
                out[t] = sum;
            }
            consumer_sync(ncons);
            if (threadIdx.x == 0) mbar_arrive(smem_addr(&empty[s]));
            reinterpret_cast<float2 *>(static_cast<float *>(L.phi) + row)[threadIdx.x] = make_float2(out[0], out[1]);
        } else if constexpr (KIND == WS_MU) {
            const float *ph = reinterpret_cast<const float *>(cur);
            constexpr int c0 = stencil_slot<Q>(0, 0);
            float out[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int x = x0 + t;
                const float p0 = ph[c0 * nx + x];
                float lap = 0.f;
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int slot = stencil_slot<Q>(Lat<Q>::cy(i), Lat<Q>::cz(i));
                    lap += float(Lat<Q>::w(i)) * (ph[slot * nx + wrap_x(x + Lat<Q>::cx(i), nx)] - p0);
                }
                lap *= 6.f;
                out[t] = float(L.P.A) * (p0 * p0 * p0 - p0) - float(L.P.kappa) * lap;
            }
            consumer_sync(ncons);
            if (threadIdx.x == 0) mbar_arrive(smem_addr(&empty[s]));
            reinterpret_cast<float2 *>(static_cast<float *>(L.mu) + row)[threadIdx.x] = make_float2(out[0], out[1]);
        } else {
            const float of = float(1.0 / L.P.tau_f), og = float(1.0 / L.P.tau_g);
            const float kf = float(1.0 - 0.5 / L.P.tau_f);
            const float g3 = float(3.0 * L.P.Gamma);
            const float *__restrict__ phif = static_cast<const float *>(L.phi);
            const float *__restrict__ muf = static_cast<const float *>(L.mu);
            float fo[NPT][Q], go[NPT][Q];
            const int xb = NPT == 1 ? (int)threadIdx.x : x0;
#pragma unroll
            for (int t = 0; t < NPT; ++t) {
                const int x = xb + t;
                const Site st = make_site(L.G, x, y, z);
                float f[Q], g[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (PULL && (wall >> i) & 1u) {
                        const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                        const float cu = float(Lat<Q>::cx(i)) * uw;
                        const float w2 = float(2.0 * Lat<Q>::w(i) * 3.0);
                        // slot i holds the local row of population opp(i)
                        const S fv = reinterpret_cast<const S *>(cur)[i * nx + x];
                        float fl;
                        if constexpr (Fmt<FMT>::DEV) fl = to_float(fv) + float(Lat<Q>::w(i)) * rho0;
                        else fl = fv;
                        f[i] = fl + w2 * rho0 * cu;
                        g[i] = fr_g<Q, FMT>(gb, nx, i, x) + w2 * php[st.n] * cu;
                    } else {
                        const int xs = PULL ? wrap_x(x - Lat<Q>::cx(i), nx) : x;
                        const S fv = reinterpret_cast<const S *>(cur)[i * nx + xs];
                        if constexpr (Fmt<FMT>::DEV) f[i] = to_float(fv) + float(Lat<Q>::w(i)) * rho0;
                        else f[i] = fv;
                        g[i] = fr_g<Q, FMT>(gb, nx, i, xs);
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
                const float *phs = reinterpret_cast<const float *>(cur + FL::f_off(nx));
                const float *mus = phs + FL::NA * nx;
                float gpx = 0.f, gpy = 0.f, gpz = 0.f, gqx = 0.f, gqy = 0.f, gqz = 0.f;
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int a = axial_slot(Lat<Q>::cy(i), Lat<Q>::cz(i));
                    float pv, mv;
                    if (a >= 0) {
                        const int xn = wrap_x(x + Lat<Q>::cx(i), nx);
                        pv = phs[a * nx + xn];
                        mv = mus[a * nx + xn];
                    } else {
                        const int kn = site_nb<Q>(st, i);
                        pv = __ldg(phif + kn);
                        mv = __ldg(muf + kn);
                    }
                    const float pm = pv * mv;
                    const float w = float(Lat<Q>::w(i));
                    if (Lat<Q>::cx(i)) { gpx += w * float(Lat<Q>::cx(i)) * pv; gqx += w * float(Lat<Q>::cx(i)) * pm; }
                    if (Lat<Q>::cy(i)) { gpy += w * float(Lat<Q>::cy(i)) * pv; gqy += w * float(Lat<Q>::cy(i)) * pm; }
                    if (Lat<Q>::cz(i)) { gpz += w * float(Lat<Q>::cz(i)) * pv; gqz += w * float(Lat<Q>::cz(i)) * pm; }
                }
                const float mu = mus[x];
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
                    fo[t][i] = fv;
                    go[t][i] = gv;
                }
                fo[t][0] = rho - fsum;
                go[t][0] = ph - gsum;
            }
            // the stage is free once every consumer has read it
            consumer_sync(ncons);
            if (threadIdx.x == 0) mbar_arrive(smem_addr(&empty[s]));
            const size_t off = row + xb;
            if constexpr (NPT == 1) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    Pop<Q, FMT>::stf(L.dst, np, i, off, fo[0][i], rho0);
                    Pop<Q, FMT>::stg(L.dst, np, i, off, go[0][i]);
                }
            } else
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S *fp = static_cast<S *>(L.dst.f) + (size_t)i * np + off;
                if constexpr (Fmt<FMT>::DEV) {
                    const float wr = float(Lat<Q>::w(i)) * rho0;
                    store2<S>(fp, fo[0][i] - wr, fo[1][i] - wr);
                    if (i == 0) {
                        *reinterpret_cast<float2 *>(L.dst.g0 + off) = make_float2(go[0][0], go[1][0]);
                    } else {
                        store2<S>(static_cast<S *>(L.dst.g) + (size_t)(i - 1) * np + off, go[0][i], go[1][i]);
                    }
                } else {
                    store2<S>(fp, fo[0][i], fo[1][i]);
                    store2<S>(static_cast<S *>(L.dst.g) + (size_t)i * np + off, go[0][i], go[1][i]);
                }
            }
        }
    }
}

template <int Q, int FMT>
struct WsRowLaunchers {
    using S = typename Fmt<FMT>::S;
    static constexpr int kMaxSmem = 200 * 1024;
    // stages per block: the update takes as many as fit (one block per SM);
    // the lighter phi and mu passes take two, so that two blocks (two
    // producer warps issuing bulk copies) share an SM
    template <int KIND>
    static int nst(int nx) {
        const unsigned sb = FullRowLayout<Q, FMT, KIND>::stage(nx);
        const int n = (int)(kMaxSmem / sb);
        if (KIND != WS_UPDATE) return n >= 2 ? 2 : n;
        return n >= 4 ? 4 : (n >= 3 ? 3 : (n >= 2 ? 2 : n));
    }
    static bool usable(const Geo &G) {
        if (G.device == FRE_FOUR_ROLLER) return false;
        if ((G.np * sizeof(S)) % 16 != 0 || (G.nx * sizeof(S)) % 16 != 0 || (G.nx * 4) % 16 != 0) return false;
        if (G.nx < 64 || G.nx > 512 || G.nx % 64 != 0) return false;
        return nst<WS_UPDATE>(G.nx) >= 2;
    }
    template <int KIND, bool PULL, int NST>
    static void launch(const Launch &L) {
        // the update keeps one node per consumer thread (more warps in
        // flight); the phi and mu passes take adjacent node pairs
        constexpr int NPT = KIND == WS_UPDATE ? 1 : 2;
        const int nx = L.G.nx;
        const int nu = L.G.ny * L.G.nz;
        const size_t smem = (size_t)NST * FullRowLayout<Q, FMT, KIND>::stage(nx);
        auto fn = k_wsrow<Q, FMT, KIND, PULL, NST, NPT>;
        static bool attr = false;
        if (!attr) {
            attr = true;
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        }
        const int threads = nx / NPT + 32;
        const int g = std::min(nu, PipeLaunchers<Q, FMT>::sms() *
                                       PipeLaunchers<Q, FMT>::blocks_per_sm((const void *)fn, threads, smem));
        fn<<<g, threads, smem, L.stream>>>(L, nu);
    }
    template <int KIND, bool PULL>
    static void run(const Launch &L) {
        switch (nst<KIND>(L.G.nx)) {
            case 4: launch<KIND, PULL, 4>(L); break;
            case 3: launch<KIND, PULL, 3>(L); break;
            default: launch<KIND, PULL, 2>(L); break;
        }
    }
    static void update(const Launch &L, bool pull) {
        if (pull) run<WS_UPDATE, true>(L);
        else run<WS_UPDATE, false>(L);
    }
    static void phi(const Launch &L, bool pull) {
        if (pull) run<WS_PHI, true>(L);
        else run<WS_PHI, false>(L);
    }
    static void mu(const Launch &L) { run<WS_MU, true>(L); }
};

}  // namespace fre

namespace fre {

// All kernels of one lattice and storage format.
template <int Q, int FMT>
const KernelSet *kernel_set_ws() {
    using GL = Launchers<Q, FMT>;
    if constexpr (FMT == FRE_FP64) {
        return kernel_set<Q, FMT>();
    } else {
        using WL = WsLaunchers<Q, FMT>;
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, WsEntry<Q, FMT>::width, WL::phi,
                                     WL::mu, WL::update, WsRowLaunchers<Q, FMT>::usable,
                                     WsRowLaunchers<Q, FMT>::update, WsRowLaunchers<Q, FMT>::phi,
                                     WsRowLaunchers<Q, FMT>::mu};
        return &ks;
    }
}

}  // namespace fre
