// Staging helpers of the chunked row kernels (k_ws): one work unit is a
// chunk of W consecutive x of one row (y, z).  The q pulled rows of f and
// g (shifted in y and z by -c_i) and the phi and mu rows of the stencil
// neighbourhood are staged into shared memory with 16-byte periodic halos
// in x, so the x part of each shift is a plain offset into the staged row.
#pragma once

#include "fre_kernels.cuh"

namespace fre {

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
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
// f / g rows.  f of slot i (a wall slot holds population opp(i)); `ref` is
// the reference the 16-bit formats add back (the fr_j of the stored row).
template <int Q, int FMT>
__device__ __forceinline__ float row_f(const unsigned char *fbase, int W, int i, int xl, float ref) {
    using S = typename Fmt<FMT>::S;
    using CL = ChunkLayout<Q, FMT>;
    const S v = reinterpret_cast<const S *>(fbase + i * CL::rw_s(W))[CL::HS + xl];
    if constexpr (Fmt<FMT>::DEV) return to_float(v) + ref;
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

// work unit: the chunk [x0, x0 + W) of row (y, z)
struct Unit {
    int y, z, x0;
    size_t row;  // global index of (0, y, z)
};

// The per-node kernels of one lattice (the FP64 format runs these alone).
template <int Q, int FMT>
const KernelSet *kernel_set() {
    using GL = Launchers<Q, FMT>;
    static const KernelSet ks = {GL::phi, GL::ghost, GL::mu, GL::update, GL::obs, GL::macro, GL::pull_plane,
                                 GL::load_plane, GL::set_phi, GL::init_eq, GL::mei_prep, GL::mei_iter,
                                 GL::mei_final, nullptr, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, nullptr};
    return &ks;
}

}  // namespace fre
