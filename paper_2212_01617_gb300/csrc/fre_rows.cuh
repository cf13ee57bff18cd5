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

// Row layout of staged populations: f rows then g rows; in 16-bit formats
// the g0 row is FP32 and sits after the 16-bit rows.
template <int Q, int FMT>
struct RowLayout {
    using S = typename Fmt<FMT>::S;
    static constexpr bool DEV = Fmt<FMT>::DEV;
    __host__ __device__ static size_t pop_bytes(int nx) {
        return DEV ? (size_t)(2 * Q - 1) * nx * sizeof(S) + (size_t)nx * 4 : (size_t)2 * Q * nx * sizeof(S);
    }
    __host__ __device__ static size_t field_off(int nx) { return (pop_bytes(nx) + 127) / 128 * 128; }
    __host__ __device__ static size_t total_bytes(int nx, int n_field_rows) {
        return field_off(nx) + (size_t)n_field_rows * nx * 4;
    }
};

// Issue the cp.async copies of `nrows` rows described by (src, dst, bytes):
// warp w copies rows w, w + nwarps, ...; its lanes take the 16-byte chunks.
__device__ __forceinline__ void stage_rows(const char *const *src, const unsigned *dst_off, const unsigned *bytes,
                                           int nrows, unsigned char *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < nrows; r += nw) {
        const unsigned chunks = bytes[r] >> 4;
        const char *s = src[r];
        unsigned char *d = smem + dst_off[r];
        for (unsigned c = lane; c < chunks; c += 32) cp_async16(d + 16 * c, s + 16 * c);
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

// Build the copy table of the population rows of lattice `lat` (0 f, 1 g)
// for row (y, z).  Wall links stage the local row of the opposite
// population.  Returns the wall-link mask.
template <int Q, int FMT>
__device__ unsigned pop_table(const Launch &L, const Buf &b, int lat, int y, int z, bool pull, const char **src,
                              unsigned *dst, unsigned *bytes, int base_slot) {
    using S = typename Fmt<FMT>::S;
    const int nx = L.G.nx;
    unsigned wall = 0;
    for (int i = 0; i < Q; ++i) {
        int ys, zs, pi = i;
        if (!src_row<Q>(L.G, y, z, i, pull, ys, zs)) {
            wall |= 1u << i;
            ys = y;
            zs = z;
            pi = Lat<Q>::opp(i);
        }
        const size_t row = ((size_t)zs * L.G.ny + ys) * nx;
        const int slot = base_slot + i;
        if (lat == 0) {
            src[slot] = static_cast<const char *>(b.f) + ((size_t)pi * L.G.np + row) * sizeof(S);
            dst[slot] = (unsigned)((size_t)i * nx * sizeof(S));
            bytes[slot] = (unsigned)(nx * sizeof(S));
        } else if (!Fmt<FMT>::DEV) {
            src[slot] = static_cast<const char *>(b.g) + ((size_t)pi * L.G.np + row) * sizeof(S);
            dst[slot] = (unsigned)((size_t)(Q + i) * nx * sizeof(S));
            bytes[slot] = (unsigned)(nx * sizeof(S));
        } else if (pi == 0) {
            src[slot] = reinterpret_cast<const char *>(b.g0 + row);
            dst[slot] = (unsigned)((size_t)(2 * Q - 1) * nx * sizeof(S));
            bytes[slot] = (unsigned)(nx * 4);
        } else {
            src[slot] = static_cast<const char *>(b.g) + ((size_t)(pi - 1) * L.G.np + row) * sizeof(S);
            // slot i of the 16-bit g rows; i = 0 can only carry the g0 row
            dst[slot] = (unsigned)((size_t)(Q + i - 1) * nx * sizeof(S));
            bytes[slot] = (unsigned)(nx * sizeof(S));
        }
    }
    return wall;
}

// Read population i of f / g at x from the staged rows.  fbase points at
// the f rows, gbase at the g rows (Q rows of the storage type; in 16-bit
// formats rows 1..Q-1 come first and the FP32 g0 row last).
template <int Q, int FMT>
__device__ __forceinline__ float row_f(const unsigned char *fbase, int nx, int i, int xs, float rho0) {
    using S = typename Fmt<FMT>::S;
    const S v = reinterpret_cast<const S *>(fbase)[(size_t)i * nx + xs];
    if constexpr (Fmt<FMT>::DEV) return to_float(v) + float(Lat<Q>::w(i)) * rho0;
    else return v;
}
template <int Q, int FMT>
__device__ __forceinline__ float row_g(const unsigned char *gbase, int nx, int i, int xs) {
    using S = typename Fmt<FMT>::S;
    if constexpr (Fmt<FMT>::DEV) {
        if (i == 0) return reinterpret_cast<const float *>(gbase + (size_t)(Q - 1) * nx * sizeof(S))[xs];
        return to_float(reinterpret_cast<const S *>(gbase)[(size_t)(i - 1) * nx + xs]);
    } else {
        return reinterpret_cast<const S *>(gbase)[(size_t)i * nx + xs];
    }
}

// ----------------------------------------------------------- phi pass

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kRowThreads) k_phi_rows(Launch L) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ const char *tsrc[2 * 19];
    __shared__ unsigned tdst[2 * 19], tbytes[2 * 19];
    __shared__ unsigned wall_s;
    const int nx = L.G.nx;
    const int r = blockIdx.x;
    const int y = r % L.G.ny, z = r / L.G.ny;
    using S = typename Fmt<FMT>::S;
    const unsigned goff = (unsigned)((size_t)Q * nx * sizeof(S));  // start of the g rows in the full layout
    if (threadIdx.x == 0) {
        wall_s = pop_table<Q, FMT>(L, L.src, 1, y, z, PULL, tsrc, tdst, tbytes, 0);
        for (int i = 0; i < Q; ++i) tdst[i] -= goff;  // only the g rows are staged here
    }
    __syncthreads();
    stage_rows(tsrc, tdst, tbytes, Q, sm);
    cp_async_wait_all();
    __syncthreads();
    const unsigned wall = wall_s;
    const float *php = static_cast<const float *>(L.phi_prev);
    float *phi = static_cast<float *>(L.phi);
    const size_t row = (size_t)r * nx;
    for (int p = threadIdx.x; p < nx / 2; p += blockDim.x) {
        float out[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = 2 * p + k;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float gi;
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                    gi = row_g<Q, FMT>(sm, nx, i, x) + float(2.0 * Lat<Q>::w(i) * 3.0) * php[row + x] *
                                                           float(Lat<Q>::cx(i)) * uw;
                } else {
                    const int xs = PULL ? wrapi(x - Lat<Q>::cx(i), nx) : x;
                    gi = row_g<Q, FMT>(sm, nx, i, xs);
                }
                s += gi;
            }
            out[k] = s;
        }
        reinterpret_cast<float2 *>(phi + row)[p] = make_float2(out[0], out[1]);
    }
}

// ------------------------------------------------------------ mu pass

template <int Q>
__global__ void __launch_bounds__(kRowThreads) k_mu_rows(Launch L) {
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int NS = n_stencil_rows<Q>();
    __shared__ const char *tsrc[NS];
    __shared__ unsigned tdst[NS], tbytes[NS];
    const int nx = L.G.nx;
    const int r = blockIdx.x;
    const int y = r % L.G.ny, z = r / L.G.ny;
    const float *phi = static_cast<const float *>(L.phi);
    if (threadIdx.x < NS) {
        const int k = threadIdx.x;
        const int cy = (Lat<Q>::D == 2 ? k : k % 3) - 1, cz = Lat<Q>::D == 2 ? 0 : k / 3 - 1;
        int yn = y + cy;
        yn = (L.G.device == FRE_SHEAR) ? (yn < 0 ? 0 : (yn >= L.G.ny ? L.G.ny - 1 : yn)) : wrapi(yn, L.G.ny);
        const int zn = wrapi(z + cz, L.G.nz);
        tsrc[k] = reinterpret_cast<const char *>(phi + ((size_t)zn * L.G.ny + yn) * nx);
        tdst[k] = (unsigned)((size_t)k * nx * 4);
        tbytes[k] = (unsigned)(nx * 4);
    }
    __syncthreads();
    stage_rows(tsrc, tdst, tbytes, NS, sm);
    cp_async_wait_all();
    __syncthreads();
    const float *ph = reinterpret_cast<const float *>(sm);
    float *mu = static_cast<float *>(L.mu) + (size_t)r * nx;
    const float A = float(L.P.A), kap = float(L.P.kappa);
    constexpr int c0 = stencil_slot<Q>(0, 0);
    for (int p = threadIdx.x; p < nx / 2; p += blockDim.x) {
        float out[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = 2 * p + k;
            const float p0 = ph[c0 * nx + x];
            float lap = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int slot = stencil_slot<Q>(Lat<Q>::cy(i), Lat<Q>::cz(i));
                lap += float(Lat<Q>::w(i)) * (ph[slot * nx + wrapi(x + Lat<Q>::cx(i), nx)] - p0);
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
__global__ void __launch_bounds__(kRowThreads) k_update_rows(Launch L) {
    using S = typename Fmt<FMT>::S;
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int NS = n_stencil_rows<Q>();
    constexpr int NR = 2 * Q + 2 * NS;
    __shared__ const char *tsrc[NR];
    __shared__ unsigned tdst[NR], tbytes[NR];
    __shared__ unsigned wall_s;
    const int nx = L.G.nx;
    const int r = blockIdx.x;
    const int y = r % L.G.ny, z = r / L.G.ny;
    const size_t foff = RowLayout<Q, FMT>::field_off(nx);
    if (threadIdx.x == 0) {
        unsigned w = pop_table<Q, FMT>(L, L.src, 0, y, z, PULL, tsrc, tdst, tbytes, 0);
        pop_table<Q, FMT>(L, L.src, 1, y, z, PULL, tsrc, tdst, tbytes, Q);
        wall_s = w;
    }
    if (threadIdx.x < 2 * NS) {
        const int k = threadIdx.x % NS, fld = threadIdx.x / NS;  // fld 0: phi, 1: mu
        const int cy = (Lat<Q>::D == 2 ? k : k % 3) - 1, cz = Lat<Q>::D == 2 ? 0 : k / 3 - 1;
        int yn = y + cy;
        yn = (L.G.device == FRE_SHEAR) ? (yn < 0 ? 0 : (yn >= L.G.ny ? L.G.ny - 1 : yn)) : wrapi(yn, L.G.ny);
        const int zn = wrapi(z + cz, L.G.nz);
        const float *base = static_cast<const float *>(fld ? L.mu : L.phi);
        const int slot = 2 * Q + fld * NS + k;
        tsrc[slot] = reinterpret_cast<const char *>(base + ((size_t)zn * L.G.ny + yn) * nx);
        tdst[slot] = (unsigned)(foff + (size_t)(fld * NS + k) * nx * 4);
        tbytes[slot] = (unsigned)(nx * 4);
    }
    __syncthreads();
    stage_rows(tsrc, tdst, tbytes, NR, sm);
    cp_async_wait_all();
    __syncthreads();

    const unsigned wall = wall_s;
    const unsigned char *gb = sm + (size_t)Q * nx * sizeof(S);
    const float *phs = reinterpret_cast<const float *>(sm + foff);
    const float *mus = phs + (size_t)NS * nx;
    const float *php = static_cast<const float *>(L.phi_prev);
    const float rho0 = float(L.P.rho0);
    const float of = float(1.0 / L.P.tau_f), og = float(1.0 / L.P.tau_g);
    const float kf = float(1.0 - 0.5 / L.P.tau_f);
    const float g3 = float(3.0 * L.P.Gamma);
    const size_t row = (size_t)r * nx;
    const long long np = L.G.np;
    constexpr int c0 = stencil_slot<Q>(0, 0);

    for (int p = threadIdx.x; p < nx / 2; p += blockDim.x) {
        float fs[2][Q], gs[2][Q];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = 2 * p + k;
            float f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (PULL && (wall >> i) & 1u) {
                    const float uw = Lat<Q>::cy(i) > 0 ? float(-L.G.uwall) : float(L.G.uwall);
                    const float cu = float(Lat<Q>::cx(i)) * uw;
                    const float w2 = float(2.0 * Lat<Q>::w(i) * 3.0);
                    // slot i holds the local row of population opp(i)
                    const int o = Lat<Q>::opp(i);
                    float fo, go;
                    if constexpr (Fmt<FMT>::DEV) {
                        fo = to_float(reinterpret_cast<const S *>(sm)[(size_t)i * nx + x]) +
                             float(Lat<Q>::w(o)) * rho0;
                    } else {
                        fo = reinterpret_cast<const S *>(sm)[(size_t)i * nx + x];
                    }
                    go = row_g<Q, FMT>(gb, nx, i, x);
                    f[i] = fo + w2 * rho0 * cu;
                    g[i] = go + w2 * php[row + x] * cu;
                } else {
                    const int xs = PULL ? wrapi(x - Lat<Q>::cx(i), nx) : x;
                    f[i] = row_f<Q, FMT>(sm, nx, i, xs, rho0);
                    g[i] = row_g<Q, FMT>(gb, nx, i, xs);
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
                const int xn = wrapi(x + Lat<Q>::cx(i), nx);
                const float pv = phs[slot * nx + xn];
                const float pm = pv * mus[slot * nx + xn];
                const float w = float(Lat<Q>::w(i));
                if (Lat<Q>::cx(i)) { gpx += w * float(Lat<Q>::cx(i)) * pv; gqx += w * float(Lat<Q>::cx(i)) * pm; }
                if (Lat<Q>::cy(i)) { gpy += w * float(Lat<Q>::cy(i)) * pv; gqy += w * float(Lat<Q>::cy(i)) * pm; }
                if (Lat<Q>::cz(i)) { gpz += w * float(Lat<Q>::cz(i)) * pv; gqz += w * float(Lat<Q>::cz(i)) * pm; }
            }
            const float mu = mus[c0 * nx + x];
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
        const size_t off = row + 2 * p;
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

template <int Q, int FMT>
struct RowLaunchers {
    using S = typename Fmt<FMT>::S;
    static size_t smem_phi(int nx) { return RowLayout<Q, FMT>::pop_bytes(nx) - (size_t)Q * nx * sizeof(S); }
    static size_t smem_mu(int nx) { return (size_t)n_stencil_rows<Q>() * nx * 4; }
    static size_t smem_update(int nx) { return RowLayout<Q, FMT>::total_bytes(nx, 2 * n_stencil_rows<Q>()); }

    static bool usable(const Geo &G) {
        if (G.device == FRE_FOUR_ROLLER) return false;
        if ((G.nx * sizeof(S)) % 16 != 0 || G.nx % 2 != 0) return false;
        if ((G.np * sizeof(S)) % 16 != 0) return false;
        return smem_update(G.nx) <= 200 * 1024;
    }
    static bool configure() {
        // opt in to the large dynamic shared memory once per process
        static bool done = false;
        static bool ok = true;
        if (!done) {
            done = true;
            const int mx = 200 * 1024;
            ok &= cudaFuncSetAttribute(k_phi_rows<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_phi_rows<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_mu_rows<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_rows<Q, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
            ok &= cudaFuncSetAttribute(k_update_rows<Q, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess;
        }
        return ok;
    }
    static void phi(const Launch &L, bool pull) {
        const unsigned rows = (unsigned)(L.G.ny * L.G.nz);
        if (pull) k_phi_rows<Q, FMT, true><<<rows, kRowThreads, smem_phi(L.G.nx), L.stream>>>(L);
        else k_phi_rows<Q, FMT, false><<<rows, kRowThreads, smem_phi(L.G.nx), L.stream>>>(L);
    }
    static void mu(const Launch &L) {
        const unsigned rows = (unsigned)(L.G.ny * L.G.nz);
        k_mu_rows<Q><<<rows, kRowThreads, smem_mu(L.G.nx), L.stream>>>(L);
    }
    static void update(const Launch &L, bool pull) {
        const unsigned rows = (unsigned)(L.G.ny * L.G.nz);
        if (pull) k_update_rows<Q, FMT, true><<<rows, kRowThreads, smem_update(L.G.nx), L.stream>>>(L);
        else k_update_rows<Q, FMT, false><<<rows, kRowThreads, smem_update(L.G.nx), L.stream>>>(L);
    }
};

template <int Q, int FMT>
struct RowEntry {
    static bool usable(const Geo &G) { return RowLaunchers<Q, FMT>::usable(G) && RowLaunchers<Q, FMT>::configure(); }
};

// All kernels of one lattice and storage format.
template <int Q, int FMT>
const KernelSet *kernel_set() {
    using GL = Launchers<Q, FMT>;
    if constexpr (FMT == FRE_FP64) {
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, nullptr, nullptr, nullptr, nullptr};
        return &ks;
    } else {
        using RL = RowLaunchers<Q, FMT>;
        static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                     GL::load_plane, GL::set_phi, GL::init_eq, RowEntry<Q, FMT>::usable, RL::phi,
                                     RL::mu, RL::update};
        return &ks;
    }
}

}  // namespace fre
