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

#include <type_traits>

#include "fre_pipe.cuh"

namespace fre {

__device__ __forceinline__ void mbar_init_count(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// expect `bytes` more transaction bytes in the current phase, without arriving
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait with a suspend hint (the warp sleeps in hardware instead of
// spinning); false once limit_ns have passed (2 s; a few ms under
// FRE_FLAG_TEST_PIPELINE_STALL).
__device__ __forceinline__ bool mbar_wait_hint(unsigned bar, unsigned parity, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    while (true) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(1000000u)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
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
    pdl_wait();

    if (producer) {
        // ------------------------------------------------------ producer warp
        // test of the timeout path: no copies are issued, so every consumer
        // wait on `full` runs out and the block leaves with an error code
        if (L.stall) return;
        const int lane = threadIdx.x - ncons;
        int k = 0;
        for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
            const int s = k % NST;
            if (k >= NST) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_hint(smem_addr(&empty[s]), (unsigned)(((k / NST) - 1) & 1), L.wait_ns);
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
    const float rho0 = L.F.rho0;
    int k = 0;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
        const int s = k % NST;
        unsigned char *cur = sm + s * stage_bytes;
        const bool ok = mbar_wait_hint(smem_addr(&full[s]), (unsigned)((k / NST) & 1), L.wait_ns);
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
                    const float uw = Lat<Q>::cy(i) > 0 ? -L.F.uwall : L.F.uwall;
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
                L.F.A * (p0 * p0 * p0 - p0) - L.F.kappa * lap;
        } else {
            const unsigned foff = CL::field_off(W);
            const unsigned char *gb = cur + CL::g_off(W);
            const unsigned char *phs = cur + foff;
            const unsigned char *mus = cur + foff + NS * CL::rw_f(W);
            const float of = L.F.omega_f, og = L.F.omega_g;
            const float kf = L.F.kf;
            const float g3 = L.F.gamma3;
            constexpr int c0 = stencil_slot<Q>(0, 0);
            // U of this row; a pulled f_i was stored in row y - c_iy
            const float U = Fmt<FMT>::DEV ? couette_u(L, u.y) : 0.f;
            float f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? -L.F.uwall : L.F.uwall;
                    const float cu = float(Lat<Q>::cx(i)) * uw;
                    const float w2 = float(2.0 * Lat<Q>::w(i) * 3.0);
                    // slot i holds the local row of population opp(i)
                    const float fo = row_f<Q, FMT>(cur, W, i, xl, fref<Q, float>(Lat<Q>::opp(i), rho0, U));
                    const float go = row_g<Q, FMT>(gb, W, i, xl);
                    f[i] = fo + w2 * rho0 * cu;
                    g[i] = go + w2 * php[u.row + u.x0 + xl] * cu;
                } else {
                    const int xs = PULL ? xl - Lat<Q>::cx(i) : xl;
                    const float Us = PULL ? couette_u(L, u.y - Lat<Q>::cy(i)) : U;
                    f[i] = row_f<Q, FMT>(cur, W, i, xs, fref<Q, float>(i, rho0, Us));
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
                    fo[i * W + xl] = from_float<S>(f[i] - fref<Q, float>(i, rho0, U));
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
    // this block is done with its units: the next kernel may start
    pdl_trigger();
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
        LaunchShape::opt_in((const void *)fn, kMaxSmem);
        const int g = std::min(nu, LaunchShape::sms() *
                                       LaunchShape::blocks_per_sm((const void *)fn, W + 32, smem));
        launch_pdl(fn, dim3(g), dim3(W + 32), smem, L.stream, L, W, nu);
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
// shift is a modular index into the staged row.  Consumer thread t of a
// row's group updates the adjacent nodes x = 2t, 2t + 1 and stores 2-wide
// vectors (the update gives each row of a unit its own group).
//   KIND WS_PHI   : stages the q pulled g rows, writes phi
//   KIND WS_MU    : stages the phi rows of the stencil, writes mu
//   KIND WS_UPDATE: stages the 2q pulled f and g rows; the phi/mu stencil
//                   values come from global memory (re-read by the nine
//                   neighbouring rows, they stay in L2)

// Work unit of the full-row kernels: R consecutive rows y0 .. y0 + R - 1 of
// one z plane (R = 2 where a row is shorter than 2 KB, so that every bulk
// copy moves at least 2 KB: the copy engine's rate of operations, not HBM,
// bounds short copies).  The R rows of a population are contiguous in
// memory and staged by one copy unless the pull offset wraps or meets a
// wall; the phi / mu stencil rows of one z plane are one copy of R + 2 rows
// (y0 - 1 .. y0 + R) unless they wrap or are clamped at a wall.
template <int Q, int FMT, int KIND, int R>
struct RowsLayout {
    using S = typename Fmt<FMT>::S;
    static constexpr bool DEV = Fmt<FMT>::DEV;
    static constexpr int D = Lat<Q>::D;
    // field rows: update -- phi and mu each: the cz = 0 group (R + 2 rows,
    // cy = -1 .. R) and in 3D the cz = +1 and cz = -1 groups (R rows, cy = 0);
    // mu pass -- phi: one group of R + 2 rows per cz in -1, 0, +1 (3D) or cz = 0
    static constexpr int NGRP = KIND == WS_UPDATE ? (D == 3 ? 3 : 1) : (KIND == WS_MU ? (D == 3 ? 3 : 1) : 0);
    static constexpr int NFIELD = KIND == WS_UPDATE ? (R + 2) + (D == 3 ? 2 * R : 0)
                                                    : (KIND == WS_MU ? NGRP * (R + 2) : 0);
    __host__ __device__ static unsigned rowb(int nx) { return (unsigned)(nx * sizeof(S)); }
    __host__ __device__ static unsigned fldb(int nx) { return (unsigned)(nx * 4); }
    // population rows: f slot i row r, then g
    __host__ __device__ static unsigned f_row(int nx, int i, int r) { return (unsigned)(i * R + r) * rowb(nx); }
    __host__ __device__ static unsigned g_off(int nx) { return KIND == WS_UPDATE ? Q * R * rowb(nx) : 0u; }
    __host__ __device__ static unsigned g_row(int nx, int i, int r) {
        if (DEV && i == 0) return g_off(nx) + (Q - 1) * R * rowb(nx) + (unsigned)r * fldb(nx);
        return g_off(nx) + (unsigned)((DEV ? i - 1 : i) * R + r) * rowb(nx);
    }
    __host__ __device__ static unsigned g_bytes(int nx) {
        return DEV ? (Q - 1) * R * rowb(nx) + R * fldb(nx) : Q * R * rowb(nx);
    }
    __host__ __device__ static unsigned fld_off(int nx) {
        return KIND == WS_UPDATE ? (g_off(nx) + g_bytes(nx) + 15u) / 16u * 16u : 0u;
    }
    // field row k of field `fld` (0 phi, 1 mu; the mu pass stages phi only)
    __host__ __device__ static unsigned fld_row(int nx, int fld, int k) {
        return fld_off(nx) + (unsigned)(fld * NFIELD + k) * fldb(nx);
    }
    // index k of the field row at (y0 + r + cy, z + cz)
    __host__ __device__ static constexpr int fk(int cy, int cz, int r) {
        return KIND == WS_MU ? (D == 3 ? (cz + 1) * (R + 2) : 0) + r + cy + 1
                             : (cz == 0 ? r + cy + 1 : (R + 2) + (cz > 0 ? 0 : R) + r);
    }
    // bytes that arrive per stage, and the stage extent
    __host__ __device__ static unsigned base_tx(int nx) {
        if (KIND == WS_MU) return NFIELD * fldb(nx);
        if (KIND == WS_UPDATE) return Q * R * rowb(nx) + g_bytes(nx) + 2 * NFIELD * fldb(nx);
        return g_bytes(nx);
    }
    __host__ __device__ static unsigned base_bytes(int nx) {
        if (KIND == WS_UPDATE) return fld_off(nx) + 2 * NFIELD * fldb(nx);
        return base_tx(nx);
    }
    __host__ __device__ static unsigned tx_bytes(int nx) { return base_tx(nx); }
    __host__ __device__ static unsigned bytes(int nx) { return base_bytes(nx); }
    __host__ __device__ static unsigned stage(int nx) { return (bytes(nx) + 127u) / 128u * 128u; }
    // copy groups issued by the producer lanes
    __host__ __device__ static constexpr int ngroups() {
        return KIND == WS_UPDATE ? 2 * Q + 2 * NGRP : (KIND == WS_PHI ? Q : NGRP);
    }
};



// Two adjacent nodes per consumer thread: FP32 arithmetic on packed pairs
// (the paired add / multiply / fused multiply-add of sm_100 and later).
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// acc + c a for a lattice component c in {-1, 0, 1} (folded after unrolling)
__device__ __forceinline__ float2 acc_c(float2 acc, float2 a, int c) {
    return c > 0 ? add2(acc, a) : (c < 0 ? sub2(acc, a) : acc);
}
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// row[x], row[x + 1] for even x (one aligned vector load)
__device__ __forceinline__ float2 ld_pair(const float *row, int x) { return *reinterpret_cast<const float2 *>(row + x); }
__device__ __forceinline__ float2 ld_pair(const __half *row, int x) {
    return __half22float2(*reinterpret_cast<const __half2 *>(row + x));
}
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16 *row, int x) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(row + x));
}
// row[xa], row[xb]
template <typename S>
__device__ __forceinline__ float2 ld_two(const S *row, int xa, int xb) {
    return make_float2(to_f(row[xa]), to_f(row[xb]));
}
// the pulled pair of one staged row: x0, x0 + 1 shifted by -cx (|cx| <= 1)
// with the periodic wrap; x0 even and 0 <= x0 <= nx - 2, so only x0 - 1 and
// x0 + 2 can leave the row
template <typename S>
__device__ __forceinline__ float2 ld_shift(const S *row, int x0, int cx, int nx) {
    if (cx == 0) return ld_pair(row, x0);
    if (cx > 0) return ld_two(row, x0 == 0 ? nx - 1 : x0 - 1, x0);
    return ld_two(row, x0 + 1, x0 + 2 == nx ? 0 : x0 + 2);
}
// start the line holding *p toward L1 (no register waits for it)
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void st_pair(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ float2 st_pair(__half *p, float2 v) {
    const __half2 h = __float22half2_rn(v);
    *reinterpret_cast<__half2 *>(p) = h;
    return __half22float2(h);
}
__device__ __forceinline__ float2 st_pair(__nv_bfloat16 *p, float2 v) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    *reinterpret_cast<__nv_bfloat162 *>(p) = h;
    return __bfloat1622float2(h);
}


// populations whose c_y has the sign of sy, as a bit mask
template <int Q>
__host__ __device__ constexpr unsigned cy_mask(int sy) {
    unsigned m = 0;
    for (int i = 0; i < Q; ++i)
        if (Lat<Q>::cy(i) * sy > 0) m |= 1u << i;
    return m;
}

// index of the opposite pair (i, opp(i)), i < opp(i), in the order i = 1, 2, ...
template <int Q>
__host__ __device__ constexpr int pair_index(int i) {
    int p = 0;
    for (int k = 1; k < i; ++k)
        if (Lat<Q>::opp(k) > k) ++p;
    return p;
}

// Per-row constants of the update for the 16-bit f formats, whose stored
// f is the deviation from the reference fr_i(y) (Eq. feq at rho0 and
// (U(y), 0, 0): the Couette profile of the shear device, or U = 0, the rest
// equilibrium, under FRE_FLAG_REST_REFERENCE and on the other devices).
// The update pulls deviations stored against the
// reference of their source row y - c_iy (or, on a wall link, the local
// deviation of opp(i)); d_i = d'_i + o_i is then the deviation from this
// row's reference, and the BGK step on deviations,
//   d*_i = (1 - omega) d_i + omega (feq_i - fr_i) + F_i,
// differs from the one on deviations from w_i rho0 by the constant
//   s_i = (1 - omega) o_i - omega (fr_i - w_i rho0).
// With a = 4.5 c_ix^2 - 1.5, b = 3 c_ix, fr_i(U) = w_i rho0 (1 + b U + a U^2):
//   o_i = w_i rho0 (b e + a (2 U + e) e),   e = U(y - c_iy) - U(y);
//   o_i = w_i rho0 6 c_ix (u_w,i - U)        on a wall link (the local
//         opp(i) plus the moving-wall term 2 w_i rho0 (c_i . u_w) / cs^2).
// Entries, each a pair (v, v): 0 sum_i o_i; 1, 2, 3 the momentum rho0 U e_x
// + sum_i c_i o_i; 4 s_0 (not read: the update closes f*_0 by the mass);
// 5 unused; 6 + 2p, 7 + 2p the parts of s_i even
// and odd in c_i of opposite pair p, (s_i + s_opp(i)) / 2 and
// (s_i - s_opp(i)) / 2.  Lane l of the calling warp takes population l.
// What couette_consts needs of the producer lane's population, computed
// once per block: the lookups by a run-time direction index (velocity,
// weight, opposite, pair slot) would otherwise be redone for every row, as
// the mbarrier waits keep the compiler from hoisting them.
struct CoLane {
    float wr, cx, cy, cz, a, b, uwl;
    int ciy, jl, slot;  // c_iy; lane of opp(i); output entry of its pair (-1: none)
};
template <int Q>
__device__ __forceinline__ CoLane co_lane(const Launch &L, int lane) {
    CoLane c;
    const int i = lane < Q ? lane : 0;
    c.ciy = Lat<Q>::cy(i);
    c.cx = float(Lat<Q>::cx(i));
    c.cy = float(c.ciy);
    c.cz = float(Lat<Q>::cz(i));
    c.wr = lane < Q ? float(Lat<Q>::w(i)) * L.F.rho0 : 0.f;
    c.a = 4.5f * c.cx * c.cx - 1.5f;
    c.b = 3.f * c.cx;
    c.uwl = c.ciy > 0 ? -L.F.uwall : L.F.uwall;
    c.jl = lane < Q ? Lat<Q>::opp(i) : lane;
    c.slot = (lane >= 1 && lane < Q && Lat<Q>::opp(i) > i) ? 6 + 2 * pair_index<Q>(i) : -1;
    return c;
}

template <int Q, bool PULL>
__device__ __forceinline__ void couette_consts(const Launch &L, const CoLane &c, int y, float2 *out, int lane) {
    const bool shear = L.G.device == FRE_SHEAR;
    const float rho0 = L.F.rho0, om = L.F.omega_f;
    const float U = couette_u(L, y);
    float o = 0.f;
    if (PULL) {
        if (shear && ((y == 0 && c.ciy > 0) || (y == L.G.ny - 1 && c.ciy < 0))) {
            o = c.wr * 6.f * c.cx * (c.uwl - U);
        } else {
            const float e = couette_u(L, y - c.ciy) - U;
            o = c.wr * (c.b * e + c.a * (2.f * U + e) * e);
        }
    }
    const float si = (1.f - om) * o - om * c.wr * (c.b * U + c.a * U * U);
    float so = o, sx = c.cx * o, sy = c.cy * o, sz = c.cz * o;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, m);
        sx += __shfl_xor_sync(0xffffffffu, sx, m);
        sy += __shfl_xor_sync(0xffffffffu, sy, m);
        sz += __shfl_xor_sync(0xffffffffu, sz, m);
    }
    const float sj = __shfl_sync(0xffffffffu, si, c.jl);
    if (lane == 0) {
        out[0] = make_float2(so, so);
        out[1] = make_float2(rho0 * U + sx, rho0 * U + sx);
        out[2] = make_float2(sy, sy);
        out[3] = make_float2(sz, sz);
        out[4] = make_float2(si, si);
        out[5] = make_float2(0.f, 0.f);
    } else if (c.slot >= 0) {
        const float e = 0.5f * (si + sj), d = 0.5f * (si - sj);
        out[c.slot] = make_float2(e, e);
        out[c.slot + 1] = make_float2(d, d);
    }
}

// Producer: copy group gi (the phi / mu stencil rows of one z plane) of
// the unit of rows y0 .. y0 + R - 1 of plane z into the stage buf, completing
// on the mbarrier bar.
template <int Q, int FMT, int KIND, int R>
__device__ __forceinline__ void stage_field_group(const Launch &L, unsigned char *buf, unsigned bar, int gi,
                                                  int y0, int z, int nx, int ny, int nz, bool shear) {
    using FL = RowsLayout<Q, FMT, KIND, R>;
    // ---- phi / mu stencil rows of one z plane
    const int j = KIND == WS_MU ? gi : gi - 2 * Q;
    const int fld = KIND == WS_MU ? 0 : j / (FL::NGRP > 0 ? FL::NGRP : 1);
    const int grp = KIND == WS_MU ? j : j - fld * FL::NGRP;
    // mu pass groups: cz = -1, 0, +1 (3D); update: cz = 0, +1, -1
    const int cz = KIND == WS_MU ? (Lat<Q>::D == 3 ? grp - 1 : 0) : (grp == 0 ? 0 : (grp == 1 ? 1 : -1));
    const bool full_y = KIND == WS_MU || cz == 0;  // R + 2 rows with y shifts
    const int zn = wrapi(z + cz, nz);
    const float *base = static_cast<const float *>(fld ? L.mu : L.phi) + (size_t)zn * ny * nx;
    const int k0 = FL::fk(full_y ? -1 : 0, cz, 0);
    unsigned char *dst = buf + FL::fld_row(nx, fld, k0);
    if (!full_y) {
        bulk_load(dst, base + (size_t)y0 * nx, (unsigned)R * FL::fldb(nx), bar);
    } else if (y0 >= 1 && y0 + R <= ny - 1) {
        bulk_load(dst, base + (size_t)(y0 - 1) * nx, (unsigned)(R + 2) * FL::fldb(nx), bar);
    } else {
        for (int q = 0; q < R + 2; ++q) {
            int yn = y0 - 1 + q;
            yn = shear ? (yn < 0 ? 0 : (yn >= ny ? ny - 1 : yn)) : wrapi(yn, ny);
            bulk_load(dst + q * FL::fldb(nx), base + (size_t)yn * nx, FL::fldb(nx), bar);
        }
    }
}

// Producer: copy group gi (one population row set: lattice f or g, direction
// i, pulled by -c_i in y and z; wall links of the shear device take the
// local row of the opposite population) of the unit into the stage buf.
template <int Q, int FMT, int KIND, int R, bool PULL>
__device__ __forceinline__ void stage_pop_group(const Launch &L, unsigned char *buf, unsigned bar, int gi, int y0,
                                                int z, int nx, int ny, int nz, bool shear) {
    using S = typename Fmt<FMT>::S;
    using FL = RowsLayout<Q, FMT, KIND, R>;
    constexpr bool DEV = Fmt<FMT>::DEV;
    // ---- population rows: lattice lat (0 f, 1 g), direction i
    const int lat = KIND == WS_PHI ? 1 : (gi >= Q);
    const int i = KIND == WS_PHI ? gi : gi - lat * Q;
    const int cy = PULL ? Lat<Q>::cy(i) : 0, cz = PULL ? Lat<Q>::cz(i) : 0;
    const int zs = wrapi(z - cz, nz);
    // source plane of population p, its element size, smem row r
    auto plane = [&](int p) -> const char * {
        if (!lat) return static_cast<const char *>(L.src.f) + (size_t)p * L.G.np * sizeof(S);
        if (DEV && p == 0) return reinterpret_cast<const char *>(L.src.g0);
        return static_cast<const char *>(L.src.g) + (size_t)(DEV ? p - 1 : p) * L.G.np * sizeof(S);
    };
    const unsigned esz = (lat && DEV && i == 0) ? 4u : (unsigned)sizeof(S);
    const unsigned rb = (unsigned)nx * esz;
    auto smrow = [&](int r) -> unsigned { return lat ? FL::g_row(nx, i, r) : FL::f_row(nx, i, r); };
    const int ys0 = y0 - cy;
    const bool inside = ys0 >= 0 && ys0 + R - 1 <= ny - 1;
    if (inside) {
        bulk_load(buf + smrow(0), plane(i) + ((size_t)zs * ny + ys0) * nx * esz, (unsigned)R * rb, bar);
    } else {
        for (int r = 0; r < R; ++r) {
            int ys = y0 + r - cy;
            int pi = i, zr = zs;
            if (ys < 0 || ys >= ny) {
                if (shear) {
                    // wall link: the local row of the opposite population
                    ys = y0 + r;
                    zr = z;
                    pi = Lat<Q>::opp(i);
                } else {
                    ys = wrapi(ys, ny);
                }
            }
            bulk_load(buf + smrow(r), plane(pi) + ((size_t)zr * ny + ys) * nx * esz, rb, bar);
        }
    }
}

// Consumers: phi = sum of the pulled g (with the moving-wall term on wall
// links) of the rows of a unit from its stage cur; the warp releases the
// stage (mbarrier empty_bar) before it stores phi.  wall_r[r]: bit i set when
// population i of row r pulls through a shear wall.
template <int Q, int FMT, int R, int RP, bool PULL>
__device__ __forceinline__ void phi_unit(const Launch &L, const unsigned char *cur, const unsigned *wall_r, int nx,
                                         int ny, int x0, int rg, int y0, int z, unsigned empty_bar) {
    using S = typename Fmt<FMT>::S;
    using FL = RowsLayout<Q, FMT, WS_PHI, R>;
    constexpr bool DEV = Fmt<FMT>::DEV;
    const float *__restrict__ php = static_cast<const float *>(L.phi_prev);
    constexpr int RT = R / RP;  // rows of this thread's group
    float2 out[RT];
#pragma unroll
    for (int q = 0; q < RT; ++q) {
        const int r = rg + q * RP;
        const unsigned wall = wall_r[r];
        const size_t row = ((size_t)z * ny + y0 + r) * nx;
        // rows without wall links (all but the first and last of the
        // shear device) take every shift as a compile-time constant
        auto pull_sum = [&](auto walls) {
            constexpr bool WL = decltype(walls)::value;
            float2 sum = p2(0.f);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool wl = WL && Lat<Q>::cy(i) != 0 && ((wall >> i) & 1u);
                const int cx = (PULL && !wl) ? Lat<Q>::cx(i) : 0;
                float2 gv;
                if (DEV && i == 0) gv = ld_shift(reinterpret_cast<const float *>(cur + FL::g_row(nx, 0, r)), x0, cx, nx);
                else gv = ld_shift(reinterpret_cast<const S *>(cur + FL::g_row(nx, i, r)), x0, cx, nx);
                if (wl) {
                    const float uw = Lat<Q>::cy(i) > 0 ? -L.F.uwall : L.F.uwall;
                    const float w2cu = float(2.0 * Lat<Q>::w(i) * 3.0) * float(Lat<Q>::cx(i)) * uw;
                    gv = fma2(p2(w2cu), ld_pair(php + row, x0), gv);
                }
                sum = add2(sum, gv);
            }
            return sum;
        };
        out[q] = (PULL && wall != 0u) ? pull_sum(std::true_type{}) : pull_sum(std::false_type{});
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(empty_bar);
#pragma unroll
    for (int q = 0; q < RT; ++q)
        st_pair(static_cast<float *>(L.phi) + ((size_t)z * ny + y0 + rg + q * RP) * nx + x0, out[q]);
}

// Consumers: mu = A (phi^3 - phi) - kappa lap(phi) of the rows of a unit from
// the staged phi stencil rows; the warp releases the stage before it stores.
// With one row group (RP = 1) a thread takes all R rows of its node pair and
// reads every staged value it needs once (the pair at x0 and the values at
// x0 - 1 and x0 + 2 of each staged row), then sums the stencil per weight
// class: lap = 6 (w_1 S_1 + w_2 S_2 - (1 - w_0) phi), S_k the sum over the
// neighbours with |c|^2 = k.
template <int Q, int FMT, int R, int RP>
__device__ __forceinline__ void mu_unit(const Launch &L, const unsigned char *cur, int nx, int ny, int x0, int rg,
                                        int y0, int z, unsigned empty_bar) {
    using FL = RowsLayout<Q, FMT, WS_MU, R>;
    constexpr int RT = R / RP;  // rows of this thread's group
    float2 out[RT];
    if constexpr (RP == 1) {
        constexpr int NP = Lat<Q>::D == 3 ? 3 : 1;  // planes cz = -1, 0, +1 (3D)
        const int xl = x0 == 0 ? nx - 1 : x0 - 1, xr = x0 + 2 == nx ? 0 : x0 + 2;
        float2 pv[NP][R + 2];
        float lv[NP][R + 2], rv[NP][R + 2];
#pragma unroll
        for (int pz = 0; pz < NP; ++pz) {
#pragma unroll
            for (int k = 0; k < R + 2; ++k) {
                const float *rw = reinterpret_cast<const float *>(
                    cur + FL::fld_row(nx, 0, FL::fk(k - 1, NP == 3 ? pz - 1 : 0, 0)));
                pv[pz][k] = ld_pair(rw, x0);
                lv[pz][k] = rw[xl];
                rv[pz][k] = rw[xr];
            }
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(empty_bar);
        constexpr float w1 = float(Lat<Q>::D == 3 ? 1.0 / 18.0 : 1.0 / 9.0), w2 = float(1.0 / 36.0);
        constexpr float wm = float(1.0 - Lat<Q>::w(0));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 s1 = p2(0.f), s2 = p2(0.f);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
                const int pz = NP == 3 ? cz + 1 : 0, k = r + 1 + cy;
                // phi at x + c_i for the pair
                const float2 v = cx == 0 ? pv[pz][k]
                                         : (cx > 0 ? make_float2(pv[pz][k].y, rv[pz][k])
                                                   : make_float2(lv[pz][k], pv[pz][k].x));
                if (cx * cx + cy * cy + cz * cz == 1) s1 = add2(s1, v);
                else s2 = add2(s2, v);
            }
            const float2 p0 = pv[NP == 3 ? 1 : 0][r + 1];
            const float2 lap = mul2(p2(6.f), fma2(p2(w1), s1, fma2(p2(w2), s2, mul2(p2(-wm), p0))));
            // A (phi^3 - phi) - kappa lap
            out[r] = sub2(mul2(p2(L.F.A), fma2(mul2(p0, p0), p0, mul2(p2(-1.f), p0))), mul2(p2(L.F.kappa), lap));
        }
    } else {
#pragma unroll
        for (int q = 0; q < RT; ++q) {
            const int r = rg + q * RP;
            const float *c0 = reinterpret_cast<const float *>(cur + FL::fld_row(nx, 0, FL::fk(0, 0, r)));
            const float2 p0 = ld_pair(c0, x0);
            float2 lap = p2(0.f);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float *rw = reinterpret_cast<const float *>(
                    cur + FL::fld_row(nx, 0, FL::fk(Lat<Q>::cy(i), Lat<Q>::cz(i), r)));
                // stencil reads x + c, i.e. a shift by -c
                lap = fma2(p2(float(Lat<Q>::w(i))), sub2(ld_shift(rw, x0, -Lat<Q>::cx(i), nx), p0), lap);
            }
            lap = mul2(p2(6.f), lap);
            // A (phi^3 - phi) - kappa lap
            out[q] = sub2(mul2(p2(L.F.A), fma2(mul2(p0, p0), p0, mul2(p2(-1.f), p0))),
                          mul2(p2(L.F.kappa), lap));
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(empty_bar);
    }
#pragma unroll
    for (int q = 0; q < RT; ++q)
        st_pair(static_cast<float *>(L.mu) + ((size_t)z * ny + y0 + rg + q * RP) * nx + x0, out[q]);
}

// Rows of a work unit run side by side, one consumer group of nx/2 threads
// each (the kernel's RPX): the update takes all R rows of a unit at once;
// the phi and mu passes loop over them, except on rows whose half length is
// not a whole number of warps (nx a multiple of 32 but not of 64), where
// every pass takes two rows side by side so that the consumers fill whole
// warps.
template <int KIND, int R>
struct RowsPar {
    static constexpr int V = KIND == WS_UPDATE ? R : 1;
};

// NXC: the row length as a compile-time constant (every shared-memory
// offset then folds into the instruction), or 0 to take it from the launch.
// ROLL: the four-roller device (roller nodes stored as 0; its wall links
// are reflected into the roller nodes' slots by k_reflect after the update).
template <int Q, int FMT, int KIND, bool PULL, int NST, int R, int NXC, int RPX, bool ROLL = false>
__global__ void __launch_bounds__(RPX * 256 + 32, KIND == WS_UPDATE ? 1 : 2) k_wsrow(Launch L, int nunits) {
    using S = typename Fmt<FMT>::S;
    using FL = RowsLayout<Q, FMT, KIND, R>;
    constexpr bool DEV = Fmt<FMT>::DEV;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) unsigned long long full[NST], empty[NST];
    __shared__ unsigned wall_s[NST][R];
    // per-row constants of the 16-bit update (couette_consts): a ring of
    // NST + 1 slots, since a consumer warp still reads those of unit k after
    // it has released the stage of unit k, until the producer may refill
    // the stage with unit k + NST
    constexpr bool CST = DEV && KIND == WS_UPDATE;
    constexpr int NCST = CST ? 6 + (Q - 1) : 2;
    __shared__ __align__(16) float2 cst_s[CST ? NST + 1 : 1][R][NCST];
    const int nx = NXC ? NXC : L.G.nx;
    const int ny = L.G.ny, nz = L.G.nz;
    const int nyu = ny / R;  // units per z plane
    // RPX rows of a unit side by side, one group of nx/2 consumer threads
    // per row (RowsPar); thread t of a group updates x = 2t, 2t + 1
    constexpr int RP = RPX;
    static_assert(R % RP == 0, "rows side by side must divide the rows of a unit");
    const int ncons = RP * (nx / 2);
    const bool producer = threadIdx.x >= ncons;
    const unsigned stage_bytes = FL::stage(nx);
    const bool shear = L.G.device == FRE_SHEAR;
    // a stage is released by each consumer warp on its own once it has read
    // it, so the consumer warps never wait for one another
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init_count(smem_addr(&full[s]), 1);
            mbar_init_count(smem_addr(&empty[s]), (unsigned)(ncons / 32));
        }
        fence_async_smem();
    }
    __syncthreads();
    pdl_wait();

    if (producer) {
        // test of the timeout path: no copies are issued, so every consumer
        // wait on `full` runs out and the block leaves with an error code
        if (L.stall) return;
        const int lane = threadIdx.x - ncons;
        const CoLane col = co_lane<Q>(L, lane);
        int k = 0;
        for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
            const int s = k % NST;
            if (k >= NST) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_hint(smem_addr(&empty[s]), (unsigned)(((k / NST) - 1) & 1), L.wait_ns);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    if (lane == 0) atomicExch(L.err, 4);
                    break;  // the consumers then time out on `full` and leave
                }
            }
            const int y0 = (unit % nyu) * R, z = unit / nyu;
            unsigned char *buf = sm + s * stage_bytes;
            const unsigned bar = smem_addr(&full[s]);
            // wall links of each row of the unit (bit i: population i pulls
            // from beyond a shear wall: c_y > 0 on row 0, c_y < 0 on row ny - 1),
            // published before the arrival that completes with the copies
            if (lane == 0) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    wall_s[s][r] = (PULL && shear) ? ((y0 + r == 0 ? cy_mask<Q>(1) : 0u) |
                                                      (y0 + r == ny - 1 ? cy_mask<Q>(-1) : 0u))
                                                   : 0u;
                // the 16-bit update arrives once its row constants are in place
                if (CST) mbar_expect_tx(bar, FL::tx_bytes(nx));
                else mbar_expect(bar, FL::tx_bytes(nx));
            }
            __syncwarp();
            for (int gi = lane; gi < FL::ngroups(); gi += 32) {
                if (KIND != WS_PHI && (KIND == WS_MU || gi >= 2 * Q))
                    stage_field_group<Q, FMT, KIND, R>(L, buf, bar, gi, y0, z, nx, ny, nz, shear);
                else
                    stage_pop_group<Q, FMT, KIND, R, PULL>(L, buf, bar, gi, y0, z, nx, ny, nz, shear);
            }
            if constexpr (CST) {
#pragma unroll
                for (int r = 0; r < R; ++r) couette_consts<Q, PULL>(L, col, y0 + r, cst_s[k % (NST + 1)][r], lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(bar);
            }
        }
        return;
    }

    // ------------------------------------------------------------ consumers
    const float rho0 = L.F.rho0;
    const float *__restrict__ php = static_cast<const float *>(L.phi_prev);
    const long long np = L.G.np;
    const int x0 = 2 * (threadIdx.x % (nx / 2));
    const int rg = RP > 1 ? threadIdx.x / (nx / 2) : 0;  // this group's row of the unit
    int k = 0;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++k) {
        const int s = k % NST;
        const unsigned char *cur = sm + s * stage_bytes;
        // a warp whose wait timed out leaves; the producer then times out
        // on the stage it never releases, and every other wait runs out too
        const bool ok = __all_sync(0xffffffffu, mbar_wait_hint(smem_addr(&full[s]), (unsigned)((k / NST) & 1), L.wait_ns));
        if (!ok) {
            if ((threadIdx.x & 31) == 0) atomicExch(L.err, 5);
            break;
        }
        const int y0 = (unit % nyu) * R, z = unit / nyu;

        if constexpr (KIND == WS_PHI) {
            phi_unit<Q, FMT, R, RP, PULL>(L, cur, wall_s[s], nx, ny, x0, rg, y0, z, smem_addr(&empty[s]));
        } else if constexpr (KIND == WS_MU) {
            mu_unit<Q, FMT, R, RP>(L, cur, nx, ny, x0, rg, y0, z, smem_addr(&empty[s]));
        } else {
            // ---------------------------------------------------- update
            const float *__restrict__ phif = static_cast<const float *>(L.phi);
            const float *__restrict__ muf = static_cast<const float *>(L.mu);
            const float of = L.F.omega_f, og = L.F.omega_g;
            const float kf = L.F.kf;
#pragma unroll 1
            for (int r = rg; r < R; r += RP) {
                const unsigned wall = wall_s[s][r];
                const int y = y0 + r;
                const size_t row = ((size_t)z * ny + y) * nx;
                const Site st = make_site(L.G, x0, y, z);
                // four-roller: the roller (solid) nodes of the pair store 0
                // in every slot (a select, no branch); k_reflect then fills
                // the slots the next step pulls through a wall link
                const uchar2 sol = ROLL ? __ldg(reinterpret_cast<const uchar2 *>(L.G.solid + row + x0))
                                        : make_uchar2(0, 0);
                auto zs2 = [&](float2 v) -> float2 {
                    if constexpr (ROLL) return make_float2(sol.x ? 0.f : v.x, sol.y ? 0.f : v.y);
                    return v;
                };
                // store a pair; returns the values as stored (16-bit: rounded)
                auto stp = [&](S *p, float2 v) -> float2 {
                    v = zs2(v);
                    if constexpr (DEV) {
                        return st_pair(p, v);
                    } else {
                        st_pair(p, v);
                        return v;
                    }
                };
                // FP32: start the lines of the off-axis stencil values (c_y and
                // c_z both nonzero, read from global memory below) toward L1
                // before the pull phase (measured 2% on the update; the
                // latency-bound 16-bit update gained nothing from it)
                if constexpr (!DEV) {
#pragma unroll
                    for (int kk = 1; kk < Q; ++kk) {
                        if (Lat<Q>::cy(kk) == 0 || Lat<Q>::cz(kk) == 0) continue;
                        const int kn = site_nb<Q>(st, kk);
                        prefetch_l1(phif + kn);
                        prefetch_l1(muf + kn);
                    }
                }
                // With the rows of a unit side by side (RP > 1, 17 warps and
                // 96 registers per thread) the update runs in two phases, so
                // that the f and g populations are never held in registers
                // together: f (pull, moments, force, velocity, collision,
                // stores), then g (pull, phi, collision, stores).  With one
                // consumer group (168 registers) both pulls come first and the
                // stage is released before any collision.  Rows without wall
                // links (all but the first and last of the shear device) take
                // every x shift as a compile-time constant.
                constexpr bool TWO = RP > 1;
                const bool walls = PULL && wall != 0u;
                // ---- f: pulled populations (16-bit: deviations from the
                // reference of the row they were stored in)
                float2 f[Q];
                auto pull_f = [&](auto wl_t) {
                    constexpr bool WL = decltype(wl_t)::value;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const bool wl = WL && Lat<Q>::cy(i) != 0 && ((wall >> i) & 1u);
                        const int cx = (PULL && !wl) ? Lat<Q>::cx(i) : 0;
                        float2 fv = ld_shift(reinterpret_cast<const S *>(cur + FL::f_row(nx, i, r)), x0, cx, nx);
                        if constexpr (!DEV) {
                            if (wl) {
                                // the row of opp(i) at this node plus the
                                // moving-wall term 2 w_i rho0 (c_i . u_w) / cs^2
                                // (16-bit f: part of the row constants)
                                const float uw = Lat<Q>::cy(i) > 0 ? -L.F.uwall : L.F.uwall;
                                fv = add2(fv, p2(float(2.0 * Lat<Q>::w(i) * 3.0) * float(Lat<Q>::cx(i)) * uw * rho0));
                            }
                        }
                        f[i] = fv;
                    }
                };
                if (walls) pull_f(std::true_type{});
                else pull_f(std::false_type{});
                // ---- g: pulled populations (now, or after the f collision)
                float2 g[Q];
                auto pull_g = [&](auto wl_t) {
                    constexpr bool WL = decltype(wl_t)::value;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const bool wl = WL && Lat<Q>::cy(i) != 0 && ((wall >> i) & 1u);
                        const int cx = (PULL && !wl) ? Lat<Q>::cx(i) : 0;
                        float2 gv;
                        if (DEV && i == 0) gv = ld_shift(reinterpret_cast<const float *>(cur + FL::g_row(nx, 0, r)), x0, cx, nx);
                        else gv = ld_shift(reinterpret_cast<const S *>(cur + FL::g_row(nx, i, r)), x0, cx, nx);
                        if (wl) {
                            // the row of opp(i) at this node plus the
                            // moving-wall term 2 w_i phi(t-1) (c_i . u_w) / cs^2
                            const float uw = Lat<Q>::cy(i) > 0 ? -L.F.uwall : L.F.uwall;
                            const float w2cu = float(2.0 * Lat<Q>::w(i) * 3.0) * float(Lat<Q>::cx(i)) * uw;
                            gv = fma2(p2(w2cu), ld_pair(php + row, x0), gv);
                        }
                        g[i] = gv;
                    }
                };
                if constexpr (!TWO) {
                    if (walls) pull_g(std::true_type{});
                    else pull_g(std::false_type{});
                }
                // stencil values of phi and mu: F = mu grad(phi) - grad(phi mu)
                float2 gpx = p2(0.f), gpy = p2(0.f), gpz = p2(0.f), gqx = p2(0.f), gqy = p2(0.f), gqz = p2(0.f);
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (Lat<Q>::opp(i) < i) continue;
                    float2 pv[2], mv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kk = h ? Lat<Q>::opp(i) : i;
                        const int cyk = Lat<Q>::cy(kk), czk = Lat<Q>::cz(kk);
                        if (cyk == 0 || czk == 0) {
                            const float *pr = reinterpret_cast<const float *>(cur + FL::fld_row(nx, 0, FL::fk(cyk, czk, r)));
                            const float *mr = reinterpret_cast<const float *>(cur + FL::fld_row(nx, 1, FL::fk(cyk, czk, r)));
                            pv[h] = ld_shift(pr, x0, -Lat<Q>::cx(kk), nx);
                            mv[h] = ld_shift(mr, x0, -Lat<Q>::cx(kk), nx);
                        } else {
                            // off-axis rows (c_x = 0): an aligned pair in global memory
                            const int kn = site_nb<Q>(st, kk);
                            pv[h] = __ldg(reinterpret_cast<const float2 *>(phif + kn));
                            mv[h] = __ldg(reinterpret_cast<const float2 *>(muf + kn));
                        }
                    }
                    const float2 dp = sub2(pv[0], pv[1]);
                    const float2 dq = sub2(mul2(pv[0], mv[0]), mul2(pv[1], mv[1]));
                    const float w = float(Lat<Q>::w(i));
                    if (Lat<Q>::cx(i)) { gpx = fma2(p2(w * Lat<Q>::cx(i)), dp, gpx); gqx = fma2(p2(w * Lat<Q>::cx(i)), dq, gqx); }
                    if (Lat<Q>::cy(i)) { gpy = fma2(p2(w * Lat<Q>::cy(i)), dp, gpy); gqy = fma2(p2(w * Lat<Q>::cy(i)), dq, gqy); }
                    if (Lat<Q>::cz(i)) { gpz = fma2(p2(w * Lat<Q>::cz(i)), dp, gpz); gqz = fma2(p2(w * Lat<Q>::cz(i)), dq, gqz); }
                }
                const float2 mu = ld_pair(reinterpret_cast<const float *>(cur + FL::fld_row(nx, 1, FL::fk(0, 0, r))), x0);
                if (!TWO && r + RP >= R) {
                    // this warp is done with the stage
                    __syncwarp();
                    if ((threadIdx.x & 31) == 0) mbar_arrive(smem_addr(&empty[s]));
                }

                // ---- moments, force, velocity (Eq. densMoment, ordeMoment, F, veloMoment)
                float2 sf = f[0], jx = p2(0.f), jy = p2(0.f), jz = p2(0.f);
                float2 ph = TWO ? p2(0.f) : g[0];
                // 16-bit f: row constants (offsets o_i summed into the moments)
                const float4 *cst = reinterpret_cast<const float4 *>(cst_s[CST ? k % (NST + 1) : 0][r]);
                if constexpr (CST) {
                    const float4 c01 = cst[0], c23 = cst[1];
                    sf = add2(sf, make_float2(c01.x, c01.y));
                    jx = make_float2(c01.z, c01.w);
                    jy = make_float2(c23.x, c23.y);
                    jz = make_float2(c23.z, c23.w);
                }
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    sf = add2(sf, f[i]);
                    if constexpr (!TWO) ph = add2(ph, g[i]);
                    jx = acc_c(jx, f[i], Lat<Q>::cx(i));
                    jy = acc_c(jy, f[i], Lat<Q>::cy(i));
                    jz = acc_c(jz, f[i], Lat<Q>::cz(i));
                }
                // sf is rho, or rho - rho0 for deviations: in both cases the
                // density term of omega (f_eq_i [- w_i rho0])
                const float2 rho = DEV ? add2(sf, p2(rho0)) : sf;
                const float2 Fx = mul2(p2(3.f), sub2(mul2(mu, gpx), gqx));
                const float2 Fy = mul2(p2(3.f), sub2(mul2(mu, gpy), gqy));
                const float2 Fz = mul2(p2(3.f), sub2(mul2(mu, gpz), gqz));
                const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
                const float2 ux = mul2(fma2(p2(0.5f), Fx, jx), inv);
                const float2 uy = mul2(fma2(p2(0.5f), Fy, jy), inv);
                const float2 uz = mul2(fma2(p2(0.5f), Fz, jz), inv);
                const float2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
                const float2 uF = fma2(ux, Fx, fma2(uy, Fy, mul2(uz, Fz)));
                const float2 omf = p2(1.f - of), omg = p2(1.f - og);
                const float2 m15usq = mul2(p2(-1.5f), usq);
                const float2 m3uF = mul2(p2(-3.f), uF);
                const float2 gmu3 = mul2(p2(L.F.gamma3), mu);
                // collision of the g pair (i, opp(i)) (Eq. LBEg, geq) and its
                // stores; cu3 = 3 c_i.u, E = 4.5 (c_i.u)^2 - 1.5 u^2
                float2 gsum = p2(0.f);
                S *gp = static_cast<S *>(L.dst.g) + row + x0;
                auto collide_g = [&](int i, int j, float w, float2 cu3, float2 E) {
                    const float2 wg = p2(og * w);
                    const float2 Ag = mul2(wg, fma2(ph, E, gmu3));
                    const float2 Bg = mul2(mul2(wg, ph), cu3);
                    const float2 gi = fma2(omg, g[i], add2(Ag, Bg)), gj = fma2(omg, g[j], sub2(Ag, Bg));
                    if constexpr (DEV) {
                        // the rest population of g closes sum_i g*_i = phi on
                        // the values as they are stored
                        gsum = add2(gsum, add2(stp(gp + (size_t)(i - 1) * np, gi), stp(gp + (size_t)(j - 1) * np, gj)));
                    } else {
                        gsum = add2(gsum, add2(stp(gp + (size_t)i * np, gi), stp(gp + (size_t)j * np, gj)));
                    }
                };

                // ---- collision of f (Eq. bgk, feq, Fi) and stores
                const size_t off = row + x0;
                S *fp = static_cast<S *>(L.dst.f) + off;
                // the rest population closes sum_i f*_i = rho below, on the
                // values as they are stored (mass is a collision invariant;
                // its own BGK formula would drift the mass by the FP32
                // rounding of the weights every step)
                float2 fsum = p2(0.f);
                // moving populations in opposite pairs (i, opp(i)): the
                // equilibrium and the Guo term split into parts even and odd
                // in c_i that the pair shares
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (Lat<Q>::opp(i) < i) continue;
                    const int j = Lat<Q>::opp(i);
                    float2 cu = p2(0.f), cF = p2(0.f);
                    cu = acc_c(cu, ux, Lat<Q>::cx(i));
                    cu = acc_c(cu, uy, Lat<Q>::cy(i));
                    cu = acc_c(cu, uz, Lat<Q>::cz(i));
                    cF = acc_c(cF, Fx, Lat<Q>::cx(i));
                    cF = acc_c(cF, Fy, Lat<Q>::cy(i));
                    cF = acc_c(cF, Fz, Lat<Q>::cz(i));
                    const float w = float(Lat<Q>::w(i));
                    const float2 cu3 = mul2(p2(3.f), cu);
                    const float2 E = fma2(mul2(p2(1.5f), cu3), cu, m15usq);  // 4.5 cu^2 - 1.5 u^2
                    const float2 wr = p2(of * w);
                    const float2 GA = fma2(mul2(p2(3.f), cu3), cF, m3uF);
                    float2 Af, Bf;
                    if constexpr (CST) {
                        // even and odd parts of the row constants s_i, s_j
                        const float4 cab = cst[3 + pair_index<Q>(i)];
                        Af = fma2(wr, fma2(rho, E, sf), fma2(p2(kf * w), GA, make_float2(cab.x, cab.y)));
                        Bf = fma2(mul2(wr, rho), cu3, fma2(p2(3.f * kf * w), cF, make_float2(cab.z, cab.w)));
                    } else {
                        Af = fma2(wr, fma2(rho, E, sf), mul2(p2(kf * w), GA));
                        Bf = fma2(mul2(wr, rho), cu3, mul2(p2(3.f * kf * w), cF));
                    }
                    const float2 fi = fma2(omf, f[i], add2(Af, Bf)), fj = fma2(omf, f[j], sub2(Af, Bf));
                    fsum = add2(fsum, add2(stp(fp + (size_t)i * np, fi), stp(fp + (size_t)j * np, fj)));
                    if constexpr (!TWO) collide_g(i, j, w, cu3, E);
                }
                // f*_0: rho - sum, or for deviations (sum_i fr_i = rho0)
                // (rho - rho0) - sum
                stp(fp, sub2(sf, fsum));

                if constexpr (TWO) {
                    if (walls) pull_g(std::true_type{});
                    else pull_g(std::false_type{});
                    if (r + RP >= R) {
                        // this warp is done with the stage
                        __syncwarp();
                        if ((threadIdx.x & 31) == 0) mbar_arrive(smem_addr(&empty[s]));
                    }
                    // ---- phi (Eq. ordeMoment) and the collision of g
                    ph = g[0];
#pragma unroll
                    for (int i = 1; i < Q; ++i) ph = add2(ph, g[i]);
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        if (Lat<Q>::opp(i) < i) continue;
                        float2 cu = p2(0.f);
                        cu = acc_c(cu, ux, Lat<Q>::cx(i));
                        cu = acc_c(cu, uy, Lat<Q>::cy(i));
                        cu = acc_c(cu, uz, Lat<Q>::cz(i));
                        const float2 cu3 = mul2(p2(3.f), cu);
                        collide_g(i, Lat<Q>::opp(i), float(Lat<Q>::w(i)), cu3, fma2(mul2(p2(1.5f), cu3), cu, m15usq));
                    }
                }
                if constexpr (DEV) {
                    st_pair(L.dst.g0 + off, zs2(sub2(ph, gsum)));
                } else {
                    stp(gp, sub2(ph, gsum));
                }

            }
        }
    }
    // this block is done with its units: the next kernel may start
    pdl_trigger();
}

// The pulled update of the four-roller device on the row kernels (roller
// nodes stored as 0; k_reflect then writes the wall links into the roller
// nodes' slots); defined in fre_rows_roller.cu, a translation unit of its
// own.  Its phi and mu passes are the plain row kernels: the pull reads the
// reflected populations from the roller slots like any other source.
template <int Q, int FMT>
struct RollRows {
    static void update(const Launch &L);
};

template <int Q, int FMT>
struct WsRowLaunchers {
    using S = typename Fmt<FMT>::S;
    static constexpr int kMaxSmem = 225 * 1024;
    // stages per block: the update takes up to three of those that fit (one
    // block per SM on long rows); the lighter phi and mu passes take two, so
    // that two blocks (two producer warps issuing bulk copies) share an SM
    template <int KIND, int R>
    static int nst(int nx) {
        const unsigned sb = RowsLayout<Q, FMT, KIND, R>::stage(nx);
        const int lim = KIND == WS_UPDATE ? kMaxSmem : kMaxSmem / 2;
        const int n = (int)(lim / sb);
        if (KIND != WS_UPDATE) return n >= 2 ? 2 : n;
        return n >= 3 ? 3 : (n >= 2 ? 2 : n);
    }
    // two rows per unit where a staged row is shorter than 2 KB
    template <int KIND>
    static int rows_per_unit(const Geo &G, bool pull) {
        // the mu pass stages three copies per unit whatever R: four rows per
        // unit keep it off the copy engine's rate of operations
        if (KIND == WS_MU) return G.ny % 4 == 0 ? 4 : (G.ny % 2 == 0 ? 2 : 1);
        // rows of an odd number of half warps: two rows side by side always
        if (G.nx % 64 != 0) return 2;
        if (!pull || G.ny % 2 != 0) return 1;
        if (RowsLayout<Q, FMT, KIND, 1>::rowb(G.nx) >= 2048) return 1;
        return nst<KIND, 2>(G.nx) >= 2 ? 2 : 1;
    }
    // the four-roller device takes the row kernels when its wall-link table
    // is there (pulled steps; the first, in-place step runs per node)
    static bool usable(const Geo &G) {
        if (G.device == FRE_FOUR_ROLLER && !G.rlinks) return false;
        if ((G.np * sizeof(S)) % 16 != 0 || (G.nx * sizeof(S)) % 16 != 0 || (G.nx * 4) % 16 != 0) return false;
        // rows of a whole number of warps' pairs (nx a multiple of 64), or of
        // an odd number of half warps taken two rows at a time (ny even)
        if (G.nx < 64 || G.nx > 512 || G.nx % 32 != 0) return false;
        if (G.nx % 64 != 0 && (G.ny % 2 != 0 || nst<WS_UPDATE, 2>(G.nx) < 2 || nst<WS_PHI, 2>(G.nx) < 2 ||
                               nst<WS_MU, 2>(G.nx) < 2 || nst<WS_MU, 4>(G.nx) < 2))
            return false;
        return nst<WS_UPDATE, 1>(G.nx) >= 2 && nst<WS_PHI, 1>(G.nx) >= 1 && nst<WS_MU, 1>(G.nx) >= 1;
    }
    template <int KIND, bool PULL, int NST, int R, int NXC, int RPX, bool ROLL = false>
    static void launch(const Launch &L) {
        const int nx = L.G.nx;
        const int nu = (L.G.ny / R) * L.G.nz;
        const size_t smem = (size_t)NST * RowsLayout<Q, FMT, KIND, R>::stage(nx);
        auto fn = k_wsrow<Q, FMT, KIND, PULL, NST, R, NXC, RPX, ROLL>;
        LaunchShape::opt_in((const void *)fn, smem);
        const int threads = RPX * (nx / 2) + 32;
        const int g = std::min(nu, LaunchShape::sms() *
                                       LaunchShape::blocks_per_sm((const void *)fn, threads, smem));
        launch_pdl(fn, dim3(g), dim3(threads), smem, L.stream, L, nu);
    }
    // resident blocks per SM of one launch shape
    template <int KIND, bool PULL, int NST, int R, int NXC, int RPX, bool ROLL = false>
    static int resident(const Launch &L) {
        const int nx = L.G.nx;
        const size_t smem = (size_t)NST * RowsLayout<Q, FMT, KIND, R>::stage(nx);
        auto fn = k_wsrow<Q, FMT, KIND, PULL, NST, R, NXC, RPX, ROLL>;
        LaunchShape::opt_in((const void *)fn, smem);
        return LaunchShape::blocks_per_sm((const void *)fn, RPX * (nx / 2) + 32, smem);
    }
    // a third stage deepens the copy pipeline, but on short rows (few
    // consumer warps per block) it can cost a resident block: keep it only
    // where the SM holds as many blocks with it as with two
    template <int KIND, bool PULL, int R, int NXC, int RPX, bool ROLL = false>
    static void run_n(const Launch &L) {
        if (nst<KIND, R>(L.G.nx) >= 3 &&
            resident<KIND, PULL, 3, R, NXC, RPX, ROLL>(L) >= resident<KIND, PULL, 2, R, NXC, RPX, ROLL>(L))
            launch<KIND, PULL, 3, R, NXC, RPX, ROLL>(L);
        else
            launch<KIND, PULL, 2, R, NXC, RPX, ROLL>(L);
    }
    template <int KIND, bool PULL, int R>
    static void run_r(const Launch &L) {
        constexpr int RPD = RowsPar<KIND, R>::V;
        // rows of an odd number of half warps: two rows side by side
        if constexpr (RPD == 1 && R % 2 == 0) {
            if (L.G.nx % 64 != 0) {
                run_n<KIND, PULL, R, 0, 2>(L);
                return;
            }
        }
        // rows of 512 nodes (the common large-lattice case) take the
        // compile-time row length
        if (PULL && L.G.nx == 512) run_n<KIND, PULL, R, 512, RPD>(L);
        else run_n<KIND, PULL, R, 0, RPD>(L);
    }
    // four-roller device, pulled steps of the update (roller nodes stored
    // as 0; instantiated in fre_rows_roller.cu)
    template <int KIND, int R>
    static void run_r_roll(const Launch &L) {
        constexpr int RPD = RowsPar<KIND, R>::V;
        if constexpr (RPD == 1 && R % 2 == 0) {
            if (L.G.nx % 64 != 0) {
                run_n<KIND, true, R, 0, 2, true>(L);
                return;
            }
        }
        run_n<KIND, true, R, 0, RPD, true>(L);
    }
    template <int KIND>
    static void run_roll(const Launch &L) {
        if (rows_per_unit<KIND>(L.G, true) == 2) run_r_roll<KIND, 2>(L);
        else run_r_roll<KIND, 1>(L);
    }
    template <int KIND, bool PULL>
    static void run(const Launch &L) {
        if constexpr (KIND == WS_UPDATE && PULL) {
            if (L.G.device == FRE_FOUR_ROLLER) {
                RollRows<Q, FMT>::update(L);
                return;
            }
        }
        const int r = rows_per_unit<KIND>(L.G, PULL);
        if constexpr (KIND == WS_MU) {
            if (r == 4) {
                run_r<KIND, PULL, 4>(L);
                return;
            }
        }
        if (r == 2) run_r<KIND, PULL, 2>(L);
        else run_r<KIND, PULL, 1>(L);
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
                                     GL::load_plane, GL::set_phi, GL::init_eq, GL::mei_prep, GL::mei_iter,
                                     GL::mei_final, WsEntry<Q, FMT>::width, WL::phi,
                                     WL::mu, WL::update, WsRowLaunchers<Q, FMT>::usable,
                                     WsRowLaunchers<Q, FMT>::update, WsRowLaunchers<Q, FMT>::phi,
                                     WsRowLaunchers<Q, FMT>::mu, GL::reflect};
        return &ks;
    }
}

}  // namespace fre
