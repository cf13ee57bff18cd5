// Row kernels: the hot path of a time step for the shear and periodic
// devices with FP32 or 16-bit population storage.
//
// A block owns one x-row (y, z) of nx nodes.  Every source row it needs
// (the q pulled rows of f and of g, shifted in y and z by -c_i, and the phi
// and mu rows of the stencil neighbourhood) is staged into shared memory
// with 16-byte cp.async copies: wide, contiguous requests are what keeps
// HBM busy on this chip, while one scalar request per population row per
// warp is not.  The x part of each shift (and the periodic wrap in x) is
// then a modular index into the staged row.  Each thread updates pairs of
// adjacent nodes and writes 2-wide vectors.
//
// Conditions (checked on the host): device != four-roller, storage FP32,
// FP16DEV or BF16DEV, nx a multiple of 16 / sizeof(storage) elements, and
// the staged rows fit in shared memory.
#pragma once

#include "fre_kernels.cuh"

namespace fre {

constexpr int kRowThreads = 256;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// slot of the stencil row (y + cy, z + cz)
template <int Q>
__host__ __device__ constexpr int stencil_slot(int cy, int cz) {
    return Lat<Q>::D == 2 ? cy + 1 : (cy + 1) + 3 * (cz + 1);
}
template <int Q>
__host__ __device__ constexpr int n_stencil_rows() {
    return Lat<Q>::D == 2 ? 3 : 9;
}

// Shared-memory layout of one work unit: a chunk of W consecutive x of one
// row (y, z).  Each staged row holds the W chunk values plus a 16-byte halo
// on each side (H = 16 / element size elements), filled from the periodic
// neighbours in x, so a shift by c_ix is a plain offset.  f rows come first,
// then g rows (in 16-bit formats rows 1..q-1, then the FP32 g0 row), then
// the FP32 phi and mu stencil rows.
template <int Q, int FMT>
struct ChunkLayout {
    using S = typename Fmt<FMT>::S;
    static constexpr bool DEV = Fmt<FMT>::DEV;
    static constexpr int HS = 16 / (int)sizeof(S);
    __host__ __device__ static unsigned rw_s(int W) { return (unsigned)((W + 2 * HS) * sizeof(S)); }
    __host__ __device__ static unsigned rw_f(int W) { return (unsigned)((W + 8) * 4); }
    __host__ __device__ static unsigned g_off(int W) { return Q * rw_s(W); }
    // offset of the FP32 g0 row from the start of the g rows (16-bit formats)
    __host__ __device__ static unsigned g0_rel(int W) { return (Q - 1) * rw_s(W); }
    __host__ __device__ static unsigned g_bytes(int W) { return DEV ? g0_rel(W) + rw_f(W) : Q * rw_s(W); }
    __host__ __device__ static unsigned pop_bytes(int W) { return g_off(W) + g_bytes(W); }
    __host__ __device__ static unsigned field_off(int W) { return (pop_bytes(W) + 127u) / 128u * 128u; }
    __host__ __device__ static unsigned total(int W, int nfield) { return field_off(W) + nfield * rw_f(W); }
};

// One staged row: global address of its x = 0 element, smem byte offset of
// the staged row (halo included) and element size.
struct RowDesc {
    const char *src;
    unsigned dst;
    unsigned esz;
};

// Issue the cp.async copies of `nrows` staged rows for the chunk [x0, x0+W):
// warp w takes rows w, w + nwarps, ...; lane c copies 16-byte chunk c, where
// chunk 0 is the left halo, chunk C-1 the right halo.
__device__ __forceinline__ void stage_chunk(const RowDesc *rows, int nrows, unsigned char *smem, int x0, int W,
                                            int nx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < nrows; r += nw) {
        const RowDesc d = rows[r];
        const int H = 16 / (int)d.esz;
        const int C = (int)(W * d.esz / 16) + 2;
        for (int c = lane; c < C; c += 32) {
            int xg;
            if (c == 0) xg = x0 >= H ? x0 - H : nx - H;
            else if (c == C - 1) xg = (x0 + W < nx) ? x0 + W : 0;
            else xg = x0 + (c - 1) * H;
            cp_async16(smem + d.dst + 16 * c, d.src + (size_t)xg * d.esz);
        }
    }
}

// source row (ys, zs) of a pulled population, or a wall link (returns false)
template <int Q>
__device__ __forceinline__ bool src_row(const Geo &G, int y, int z, int i, bool pull, int &ys, int &zs) {
    if (!pull) {
        ys = y;
        zs = z;
        return true;
    }
    ys = y - Lat<Q>::cy(i);
    zs = wrapi(z - Lat<Q>::cz(i), G.nz);
    if (G.device == FRE_SHEAR) {
        if (ys < 0 || ys >= G.ny) return false;
    } else {
        ys = wrapi(ys, G.ny);
    }
    return true;
}

// Staged row of population i of lattice `lat` (0 f, 1 g) for the work row
// (y, z); smem offset relative to `base` (the start of this lattice's rows).
// A wall link stages the local row of the opposite population and sets
// *wall.
template <int Q, int FMT>
__device__ __forceinline__ RowDesc pop_row(const Launch &L, const Buf &b, int lat, int i, int y, int z, bool pull,
                                           int W, unsigned base, bool *wall) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    int ys, zs, pi = i;
    *wall = false;
    if (!src_row<Q>(L.G, y, z, i, pull, ys, zs)) {
        *wall = true;
        ys = y;
        zs = z;
        pi = Lat<Q>::opp(i);
    }
    const size_t row = ((size_t)zs * L.G.ny + ys) * L.G.nx;
    RowDesc d;
    if (lat == 0) {
        d.src = static_cast<const char *>(b.f) + ((size_t)pi * L.G.np + row) * sizeof(S);
        d.dst = base + i * CL::rw_s(W);
        d.esz = sizeof(S);
    } else if (!Fmt<FMT>::DEV) {
        d.src = static_cast<const char *>(b.g) + ((size_t)pi * L.G.np + row) * sizeof(S);
        d.dst = base + i * CL::rw_s(W);
        d.esz = sizeof(S);
    } else if (pi == 0) {  // only for i = 0 (opp(i) = 0 iff i = 0)
        d.src = reinterpret_cast<const char *>(b.g0 + row);
        d.dst = base + CL::g0_rel(W);
        d.esz = 4;
    } else {
        d.src = static_cast<const char *>(b.g) + ((size_t)(pi - 1) * L.G.np + row) * sizeof(S);
        d.dst = base + (i - 1) * CL::rw_s(W);
        d.esz = sizeof(S);
    }
    return d;
}

// Stencil rows (y + cy, z + cz) of a FP32 field, slot k, at smem base.
template <int Q>
__device__ __forceinline__ RowDesc field_row(const Launch &L, const float *field, int y, int z, int k, int W,
                                             unsigned base) {
    const int cy = (Lat<Q>::D == 2 ? k : k % 3) - 1, cz = Lat<Q>::D == 2 ? 0 : k / 3 - 1;
    int yn = y + cy;
    yn = (L.G.device == FRE_SHEAR) ? (yn < 0 ? 0 : (yn >= L.G.ny ? L.G.ny - 1 : yn)) : wrapi(yn, L.G.ny);
    const int zn = wrapi(z + cz, L.G.nz);
    RowDesc d;
    d.src = reinterpret_cast<const char *>(field + ((size_t)zn * L.G.ny + yn) * L.G.nx);
    d.dst = base + (unsigned)k * (unsigned)((W + 8) * 4);
    d.esz = 4;
    return d;
}

// Staged values at local x (-1 <= xl <= W).  fbase / gbase: start of the
// f / g rows.
template <int Q, int FMT>
__device__ __forceinline__ float row_f(const unsigned char *fbase, int W, int i, int xl, float rho0) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    const S v = reinterpret_cast<const S *>(fbase + i * CL::rw_s(W))[CL::HS + xl];
    if constexpr (Fmt<FMT>::DEV) return to_float(v) + float(Lat<Q>::w(i)) * rho0;
    else return v;
}
// raw staged f of slot i (a wall slot holds population opp(i))
template <int Q, int FMT>
__device__ __forceinline__ float row_f_slot(const unsigned char *fbase, int W, int i, int xl, float wr) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    const S v = reinterpret_cast<const S *>(fbase + i * CL::rw_s(W))[CL::HS + xl];
    if constexpr (Fmt<FMT>::DEV) return to_float(v) + wr;
    else return v;
}
template <int Q, int FMT>
__device__ __forceinline__ float row_g(const unsigned char *gbase, int W, int i, int xl) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    if constexpr (Fmt<FMT>::DEV) {
        if (i == 0) return reinterpret_cast<const float *>(gbase + CL::g0_rel(W))[4 + xl];
        return to_float(reinterpret_cast<const S *>(gbase + (i - 1) * CL::rw_s(W))[CL::HS + xl]);
    } else {
        return reinterpret_cast<const S *>(gbase + i * CL::rw_s(W))[CL::HS + xl];
    }
}
__device__ __forceinline__ float row_field(const unsigned char *fbase, int W, int k, int xl) {
    return reinterpret_cast<const float *>(fbase + (unsigned)k * (unsigned)((W + 8) * 4))[4 + xl];
}

// work unit of block b: chunk c of row r
struct Unit {
    int y, z, x0;
    size_t row;  // global index of (0, y, z)
};
__device__ __forceinline__ Unit unit_of(const Geo &G, int W) {
    const int nch = G.nx / W;
    const int b = blockIdx.x;
    const int r = b / nch;
    Unit u;
    u.x0 = (b - r * nch) * W;
    u.y = r % G.ny;
    u.z = r / G.ny;
    u.row = (size_t)r * G.nx;
    return u;
}

// ----------------------------------------------------------- phi pass

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kRowThreads) k_phi_rows(Launch L, int W) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ RowDesc rows[19];
    __shared__ unsigned wall_s;
    const Unit u = unit_of(L.G, W);
    if (threadIdx.x == 0) wall_s = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < Q; k += blockDim.x) {
        bool w;
        rows[k] = pop_row<Q, FMT>(L, L.src, 1, k, u.y, u.z, PULL, W, 0u, &w);
        if (w) atomicOr(&wall_s, 1u << k);
    }
    __syncthreads();
    stage_chunk(rows, Q, sm, u.x0, W, L.G.nx);
    cp_async_wait_all();
    __syncthreads();
    const unsigned wall = wall_s;
    const float *php = static_cast<const float *>(L.phi_prev);
    float *phi = static_cast<float *>(L.phi) + u.row + u.x0;
    for (int p = threadIdx.x; p < W / 2; p += blockDim.x) {
        float out[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int xl = 2 * p + k;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float gi;
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                    gi = row_g<Q, FMT>(sm, W, i, xl) +
                         float(2.0 * Lat<Q>::w(i) * 3.0) * php[u.row + u.x0 + xl] * float(Lat<Q>::cx(i)) * uw;
                } else {
                    gi = row_g<Q, FMT>(sm, W, i, PULL ? xl - Lat<Q>::cx(i) : xl);
                }
                s += gi;
            }
            out[k] = s;
        }
        reinterpret_cast<float2 *>(phi)[p] = make_float2(out[0], out[1]);
    }
}

// ------------------------------------------------------------ mu pass

template <int Q>
__global__ void __launch_bounds__(kRowThreads) k_mu_rows(Launch L, int W) {
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int NS = n_stencil_rows<Q>();
    __shared__ RowDesc rows[NS];
    const Unit u = unit_of(L.G, W);
    if (threadIdx.x < NS)
        rows[threadIdx.x] = field_row<Q>(L, static_cast<const float *>(L.phi), u.y, u.z, threadIdx.x, W, 0u);
    __syncthreads();
    stage_chunk(rows, NS, sm, u.x0, W, L.G.nx);
    cp_async_wait_all();
    __syncthreads();
    float *mu = static_cast<float *>(L.mu) + u.row + u.x0;
    const float A = float(L.P.A), kap = float(L.P.kappa);
    constexpr int c0 = stencil_slot<Q>(0, 0);
    for (int p = threadIdx.x; p < W / 2; p += blockDim.x) {
        float out[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int xl = 2 * p + k;
            const float p0 = row_field(sm, W, c0, xl);
            float lap = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int slot = stencil_slot<Q>(Lat<Q>::cy(i), Lat<Q>::cz(i));
                lap += float(Lat<Q>::w(i)) * (row_field(sm, W, slot, xl + Lat<Q>::cx(i)) - p0);
            }
            lap *= 6.f;
            out[k] = A * (p0 * p0 * p0 - p0) - kap * lap;
        }
        reinterpret_cast<float2 *>(mu)[p] = make_float2(out[0], out[1]);
    }
}

// ---------------------------------------------------------- update pass

template <typename S>
__device__ __forceinline__ void store2(S *p, float a, float b);
template <>
__device__ __forceinline__ void store2<float>(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store2<__half>(__half *p, float a, float b) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kRowThreads) k_update_rows(Launch L, int W) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int NS = n_stencil_rows<Q>();
    constexpr int NR = 2 * Q + 2 * NS;
    __shared__ RowDesc rows[NR];
    __shared__ unsigned wall_s;
    const Unit u = unit_of(L.G, W);
    const unsigned foff = CL::field_off(W);
    if (threadIdx.x == 0) wall_s = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < NR; k += blockDim.x) {
        if (k < 2 * Q) {
            const int lat = k >= Q, i = k - lat * Q;
            bool w;
            rows[k] = pop_row<Q, FMT>(L, L.src, lat, i, u.y, u.z, PULL, W, lat ? CL::g_off(W) : 0u, &w);
            if (w && !lat) atomicOr(&wall_s, 1u << i);
        } else {
            const int j = k - 2 * Q, fld = j / NS, m = j - fld * NS;  // fld 0: phi, 1: mu
            const float *base = static_cast<const float *>(fld ? L.mu : L.phi);
            rows[k] = field_row<Q>(L, base, u.y, u.z, m, W, foff + fld * NS * CL::rw_f(W));
        }
    }
    __syncthreads();
    stage_chunk(rows, NR, sm, u.x0, W, L.G.nx);
    cp_async_wait_all();
    __syncthreads();

    const unsigned wall = wall_s;
    const unsigned char *gb = sm + CL::g_off(W);
    const unsigned char *phs = sm + foff;
    const unsigned char *mus = sm + foff + NS * CL::rw_f(W);
    const float *php = static_cast<const float *>(L.phi_prev);
    const float rho0 = float(L.P.rho0);
    const float of = float(1.0 / L.P.tau_f), og = float(1.0 / L.P.tau_g);
    const float kf = float(1.0 - 0.5 / L.P.tau_f);
    const float g3 = float(3.0 * L.P.Gamma);
    const long long np = L.G.np;
    constexpr int c0 = stencil_slot<Q>(0, 0);

    for (int p = threadIdx.x; p < W / 2; p += blockDim.x) {
        float fs[2][Q], gs[2][Q];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int xl = 2 * p + k;
            float f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                    const float cu = float(Lat<Q>::cx(i)) * uw;
                    const float w2 = float(2.0 * Lat<Q>::w(i) * 3.0);
                    // slot i holds the local row of population opp(i)
                    const float fo = row_f_slot<Q, FMT>(sm, W, i, xl, float(Lat<Q>::w(Lat<Q>::opp(i))) * rho0);
                    const float go = row_g<Q, FMT>(gb, W, i, xl);
                    f[i] = fo + w2 * rho0 * cu;
                    g[i] = go + w2 * php[u.row + u.x0 + xl] * cu;
                } else {
                    const int xs = PULL ? xl - Lat<Q>::cx(i) : xl;
                    f[i] = row_f<Q, FMT>(sm, W, i, xs, rho0);
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
                fs[k][i] = fv;
                gs[k][i] = gv;
            }
            fs[k][0] = rho - fsum;
            gs[k][0] = ph - gsum;
        }
        // 2-wide stores of the node pair
        const size_t off = u.row + u.x0 + 2 * p;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            S *fp = static_cast<S *>(L.dst.f) + (size_t)i * np + off;
            if constexpr (Fmt<FMT>::DEV) {
                const float wr = float(Lat<Q>::w(i)) * rho0;
                store2<S>(fp, fs[0][i] - wr, fs[1][i] - wr);
                if (i == 0) {
                    *reinterpret_cast<float2 *>(L.dst.g0 + off) = make_float2(gs[0][0], gs[1][0]);
                } else {
                    store2<S>(static_cast<S *>(L.dst.g) + (size_t)(i - 1) * np + off, gs[0][i], gs[1][i]);
                }
            } else {
                store2<S>(fp, fs[0][i], fs[1][i]);
                store2<S>(static_cast<S *>(L.dst.g) + (size_t)i * np + off, gs[0][i], gs[1][i]);
            }
        }
    }
}

// -------------------------------------------------------------- launch

// Chunk width: 128 x per work unit when nx allows it (small shared-memory
// footprint, several blocks per SM to overlap staging with compute), else
// the whole row.  `pref` (a power of two, 0 = automatic) overrides.
inline int chunk_width(const Geo &G, int elem_bytes, int pref) {
    auto ok = [&](int W) { return W >= 2 && G.nx % W == 0 && (W * elem_bytes) % 16 == 0 && W % 2 == 0; };
    if (pref > 0 && ok(pref)) return pref;
    if (ok(128)) return 128;
    return G.nx;
}

template <int Q, int FMT>
struct RowLaunchers {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    static constexpr int kMaxSmem = 200 * 1024;
    static size_t smem_phi(int W) { return CL::g_bytes(W); }
    static size_t smem_mu(int W) { return (size_t)n_stencil_rows<Q>() * CL::rw_f(W); }
    static size_t smem_update(int W) { return CL::total(W, 2 * n_stencil_rows<Q>()); }
    static int threads(int W) {
        int t = W / 2;
        t = (t + 31) / 32 * 32;
        return t < kRowThreads ? t : kRowThreads;
    }

    static bool usable(const Geo &G, int W) {
        if (G.device == FRE_FOUR_ROLLER) return false;
        if (G.nx % 2 != 0 || (G.nx * sizeof(S)) % 16 != 0 || G.nx < 16 / (int)sizeof(S)) return false;
        if ((G.np * sizeof(S)) % 16 != 0) return false;
        if (G.nx % W != 0 || (W * sizeof(S)) % 16 != 0) return false;
        return smem_update(W) <= (size_t)kMaxSmem;
    }
    static bool configure() {
        // opt in to the large dynamic shared memory once per process
        static bool done = false;
        static bool ok = true;
        if (!done) {
            done = true;
            const int mx = kMaxSmem;
            ok &= cudaFuncSetAttribute(k_phi_rows<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_phi_rows<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_mu_rows<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_rows<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_rows<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
        }
        return ok;
    }
    static unsigned blocks(const Launch &L) { return (unsigned)((size_t)L.G.ny * L.G.nz * (L.G.nx / L.W)); }
    static void phi(const Launch &L, bool pull) {
        if (pull) k_phi_rows<Q, FMT, true><<<blocks(L), threads(L.W), smem_phi(L.W), L.stream>>>(L, L.W);
        else k_phi_rows<Q, FMT, false><<<blocks(L), threads(L.W), smem_phi(L.W), L.stream>>>(L, L.W);
    }
    static void mu(const Launch &L) { k_mu_rows<Q><<<blocks(L), threads(L.W), smem_mu(L.W), L.stream>>>(L, L.W); }
    static void update(const Launch &L, bool pull) {
        if (pull) k_update_rows<Q, FMT, true><<<blocks(L), threads(L.W), smem_update(L.W), L.stream>>>(L, L.W);
        else k_update_rows<Q, FMT, false><<<blocks(L), threads(L.W), smem_update(L.W), L.stream>>>(L, L.W);
    }
};

template <int Q, int FMT>
struct RowEntry {
    // chunk width for this geometry (0: the row kernels do not apply)
    static int width(const Geo &G, int pref) {
        const int W = chunk_width(G, (int)sizeof(typename Fmt<FMT>::S), pref);
        return (RowLaunchers<Q, FMT>::usable(G, W) && RowLaunchers<Q, FMT>::configure()) ? W : 0;
    }
};

// All kernels of one lattice and storage format.
template <int Q, int FMT>
const KernelSet *kernel_set() {
    using GL = Launchers<Q, FMT>;
    if constexpr (FMT == FRE_FP64) {
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, nullptr, nullptr, nullptr, nullptr,
                                     nullptr, nullptr, nullptr, nullptr};
        return &ks;
    } else {
        using RL = RowLaunchers<Q, FMT>;
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, RowEntry<Q, FMT>::width, RL::phi,
                                     RL::mu, RL::update, nullptr, nullptr, nullptr, nullptr};
        return &ks;
    }
}

}  // namespace fre
