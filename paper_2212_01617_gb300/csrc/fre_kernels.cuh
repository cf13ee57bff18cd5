// Kernels of the two-lattice free energy LBM time step (Simonis et al.,
// arXiv:2212.01617, Sec. 2.2-2.3, Algorithm 1), templated on the velocity
// set (Q = 9, 19) and the population storage format.
//
// Data layout (device memory, one context):
//   populations  SoA planes [q][np], node n = (z*ny + y)*nx + x (x fastest),
//                two buffers A/B (pull streaming A -> B, then swap);
//   phi, mu      one value per node in the compute type; phi in two
//                buffers (current step / previous step).
// One time step = k_phi (pull g, phi = sum g) -> [roller ghosts] -> k_mu
// (mu from the phi stencil) -> [roller ghosts] -> k_update (pull f and g,
// moments, force from the phi/mu stencils, BGK + Guo for f, BGK for g, store
// post-collision populations).  The state between steps is the
// post-collision buffer; streaming happens as the next step pulls from it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fre_internal.h"
#include "lattice.cuh"

namespace fre {

// Programmatic dependent launch (sm_90 and later).  The kernels of a time
// step are launched with launch_pdl: each may start (block scheduling,
// shared-memory and barrier set-up, reads of launch tables) while the
// kernel before it in the stream is still finishing, and waits for that
// kernel's completion and memory (griddepcontrol.wait, pdl_wait) before it
// reads or writes any field or population.  The persistent row kernels let
// their successor start once a block is done with its units (pdl_trigger);
// the others when they exit.  The wait is a no-op for a kernel launched
// without the attribute, and a kernel launched normally after one of these
// starts only when it ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       const Args &...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, fn, args...);
}

constexpr int kBlock = 256;

template <int FMT>
struct Fmt;
template <>
struct Fmt<FRE_FP64> {
    using S = double;
    using T = double;
    static constexpr bool DEV = false;
};
template <>
struct Fmt<FRE_FP32> {
    using S = float;
    using T = float;
    static constexpr bool DEV = false;
};
template <>
struct Fmt<FRE_FP16DEV> {
    using S = __half;
    using T = float;
    static constexpr bool DEV = true;
};
template <>
struct Fmt<FRE_BF16DEV> {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr bool DEV = true;
};

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__half h) { return __half2float(h); }
__device__ __forceinline__ float to_float(__nv_bfloat16 h) { return __bfloat162float(h); }
template <typename S>
__device__ __forceinline__ S from_float(float v);
template <>
__device__ __forceinline__ float from_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Reference state of the 16-bit f formats.  f is stored as the deviation
// f_i - fr_i(y) from the second-order equilibrium (Eq. feq) of density rho0
// and velocity (U(y), 0, 0).  The shear device takes the plane Couette
// profile between its walls, U(y) = u_w (2 (y + 1/2) / ny - 1), so the
// stored values carry the departure from the base flow only instead of
// spending the 16-bit mantissa on the 3 w_i rho0 c_ix U part of every
// moving population; under FRE_FLAG_REST_REFERENCE, and on the other
// devices, U = 0: the rest equilibrium w_i rho0.  U(y) = u0 + y du with u0,
// du rounded on the host.
__device__ __forceinline__ float couette_u(const Launch &L, int y) { return fmaf(float(y), L.F.du, L.F.u0); }
template <int Q, typename T>
__device__ __forceinline__ T fref(int i, T rho0, T U) {
    const T cu = T(Lat<Q>::cx(i)) * U;
    return T(Lat<Q>::w(i)) * rho0 * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * U * U);
}

// fr_i - w_i rho0: the small part of the reference, O(U), evaluated apart so
// that deviations from w_i rho0 never pass through values of size w_i
template <int Q, typename T>
__device__ __forceinline__ T eref(int i, T rho0, T U) {
    const T cu = T(Lat<Q>::cx(i)) * U;
    return T(Lat<Q>::w(i)) * rho0 * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * U * U);
}

// Population access for one buffer in a given storage format.  ldf / stf
// take rho0 and U of the row of node k (the reference of the 16-bit f
// formats; unused by the others).
template <int Q, int FMT>
struct Pop {
    using S = typename Fmt<FMT>::S;
    using T = typename Fmt<FMT>::T;

    __device__ __forceinline__ static T ldf(const Buf &b, long long np, int i, long long k, T rho0, T U) {
        const S *p = static_cast<const S *>(b.f) + (size_t)i * np + k;
        if constexpr (!Fmt<FMT>::DEV) {
            return __ldg(p);
        } else {
            return to_float(__ldg(p)) + fref<Q, T>(i, rho0, U);
        }
    }
    __device__ __forceinline__ static T ldg(const Buf &b, long long np, int i, long long k) {
        if constexpr (!Fmt<FMT>::DEV) {
            return __ldg(static_cast<const S *>(b.g) + (size_t)i * np + k);
        } else {
            if (i == 0) return __ldg(b.g0 + k);
            return to_float(__ldg(static_cast<const S *>(b.g) + (size_t)(i - 1) * np + k));
        }
    }
    __device__ __forceinline__ static void stf(const Buf &b, long long np, int i, long long k, T v, T rho0, T U) {
        S *p = static_cast<S *>(b.f) + (size_t)i * np + k;
        if constexpr (!Fmt<FMT>::DEV) {
            *p = v;
        } else {
            *p = from_float<S>(v - fref<Q, T>(i, rho0, U));
        }
    }
    // 16-bit formats: f_i - w_i rho0 of a stored f (deviation d from
    // fr_i(U) plus the small part of the reference)
    __device__ __forceinline__ static T ldw(const Buf &b, long long np, int i, long long k, T rho0, T U) {
        return to_float(__ldg(static_cast<const S *>(b.f) + (size_t)i * np + k)) + eref<Q, T>(i, rho0, U);
    }
    // 16-bit formats: store f_i given as W = f_i - w_i rho0; returns W as
    // stored (the rounded deviation plus the small part of the reference)
    __device__ __forceinline__ static T stw_back(const Buf &b, long long np, int i, long long k, T W, T rho0, T U) {
        const T e = eref<Q, T>(i, rho0, U);
        const S s = from_float<S>(W - e);
        static_cast<S *>(b.f)[(size_t)i * np + k] = s;
        return to_float(s) + e;
    }
    // store and return the value as stored (16-bit formats: rounded), so
    // that the rest population can close the collision invariants on the
    // stored populations
    __device__ __forceinline__ static T stf_back(const Buf &b, long long np, int i, long long k, T v, T rho0, T U) {
        S *p = static_cast<S *>(b.f) + (size_t)i * np + k;
        if constexpr (!Fmt<FMT>::DEV) {
            *p = v;
            return v;
        } else {
            const T r = fref<Q, T>(i, rho0, U);
            const S s = from_float<S>(v - r);
            *p = s;
            return to_float(s) + r;
        }
    }
    __device__ __forceinline__ static T stg_back(const Buf &b, long long np, int i, long long k, T v) {
        if constexpr (!Fmt<FMT>::DEV) {
            static_cast<S *>(b.g)[(size_t)i * np + k] = v;
            return v;
        } else {
            if (i == 0) {
                b.g0[k] = v;
                return v;
            }
            const S s = from_float<S>(v);
            static_cast<S *>(b.g)[(size_t)(i - 1) * np + k] = s;
            return to_float(s);
        }
    }
    __device__ __forceinline__ static void stg(const Buf &b, long long np, int i, long long k, T v) {
        if constexpr (!Fmt<FMT>::DEV) {
            static_cast<S *>(b.g)[(size_t)i * np + k] = v;
        } else {
            if (i == 0) {
                b.g0[k] = v;
            } else {
                static_cast<S *>(b.g)[(size_t)(i - 1) * np + k] = from_float<S>(v);
            }
        }
    }
};

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ int node_index(const Geo &G, int x, int y, int z) {
    return (z * G.ny + y) * G.nx + x;
}

// x, y, z of node n (only used off the hot path; N < 2^31 is enforced at create)
__device__ __forceinline__ void decode(const Geo &G, int n, int &x, int &y, int &z) {
    const int nxy = G.nx * G.ny;
    z = n / nxy;
    const int r = n - z * nxy;
    y = r / G.nx;
    x = r - y * G.nx;
}

__device__ __forceinline__ bool is_solid(const Geo &G, int n) {
    return G.device == FRE_FOUR_ROLLER && G.solid[n] != 0;
}

// A node and the index deltas of its six axis neighbours, computed once per
// thread; every stencil and streaming index is then n plus up to three of
// them.  Periodic in x and z; in y periodic, except for the shear device,
// where the stencil delta across a wall is 0 (the value behind the half-way
// wall mirrors the first fluid row) and ylo/yhi flag links that enter the
// channel through the bottom/top wall.
struct Site {
    int n, x, y, z;
    int dxp, dxm, dyp, dym, dzp, dzm;
    bool ylo, yhi;
};

__device__ __forceinline__ Site make_site(const Geo &G, int x, int y, int z) {
    Site s;
    s.x = x;
    s.y = y;
    s.z = z;
    s.n = node_index(G, x, y, z);
    const int sy = G.nx, sz = G.nx * G.ny;
    s.dxp = (x == G.nx - 1) ? 1 - G.nx : 1;
    s.dxm = (x == 0) ? G.nx - 1 : -1;
    if (G.device == FRE_SHEAR) {
        s.dyp = (y == G.ny - 1) ? 0 : sy;
        s.dym = (y == 0) ? 0 : -sy;
        s.ylo = (y == 0);
        s.yhi = (y == G.ny - 1);
    } else {
        s.dyp = (y == G.ny - 1) ? (1 - G.ny) * sy : sy;
        s.dym = (y == 0) ? (G.ny - 1) * sy : -sy;
        s.ylo = s.yhi = false;
    }
    s.dzp = (z == G.nz - 1) ? (1 - G.nz) * sz : sz;
    s.dzm = (z == 0) ? (G.nz - 1) * sz : -sz;
    return s;
}

// stencil neighbour x + c_i
template <int Q>
__device__ __forceinline__ int site_nb(const Site &s, int i) {
    const int cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    return s.n + (cx > 0 ? s.dxp : (cx < 0 ? s.dxm : 0)) + (cy > 0 ? s.dyp : (cy < 0 ? s.dym : 0)) +
           (cz > 0 ? s.dzp : (cz < 0 ? s.dzm : 0));
}

// streaming source x - c_i (meaningful when the link is not a wall link)
template <int Q>
__device__ __forceinline__ int site_src(const Site &s, int i) {
    const int cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    return s.n + (cx > 0 ? s.dxm : (cx < 0 ? s.dxp : 0)) + (cy > 0 ? s.dym : (cy < 0 ? s.dyp : 0)) +
           (cz > 0 ? s.dzm : (cz < 0 ? s.dzp : 0));
}

// Streaming source x - c_i.  Returns its index when it is fluid; returns -1
// and the wall velocity at the link's wall point x - c_i/2 when it is solid.
template <int Q, typename T>
__device__ __forceinline__ int pull_source(const Geo &G, const Site &s, int i, T &uwx, T &uwy) {
    const int cy = Lat<Q>::cy(i);
    if (G.device == FRE_SHEAR) {
        if (cy > 0 && s.ylo) {
            uwx = T(-G.uwall);
            uwy = T(0);
            return -1;
        }
        if (cy < 0 && s.yhi) {
            uwx = T(G.uwall);
            uwy = T(0);
            return -1;
        }
        return site_src<Q>(s, i);
    }
    const int src = site_src<Q>(s, i);
    if (G.device == FRE_FOUR_ROLLER) {
        const int k = G.solid[src];
        if (k) {
            // the wall point in the frame of the roller: the wrapped source
            // plus c_i / 2
            const double xw = wrapi(s.x - Lat<Q>::cx(i), G.nx) + 0.5 * Lat<Q>::cx(i);
            const double yw = wrapi(s.y - cy, G.ny) + 0.5 * cy;
            uwx = T(-G.om[k] * (yw - G.rcy[k]));
            uwy = T(G.om[k] * (xw - G.rcx[k]));
            return -1;
        }
    }
    return src;
}

// Pre-collision populations of a node: pulled from the post-collision
// buffer (with half-way bounce-back and the moving-wall term
//   f_i = f*_ibar + 2 w_i rho0 (c_i . u_w)/cs^2,
//   g_i = g*_ibar + 2 w_i phi(x, t-1) (c_i . u_w)/cs^2)
// or read in place.
//
// 16-bit formats: f_i is assembled from its deviation from w_i rho0, W_i =
// d_i + (fr_i - w_i rho0), all small numbers, and *wsum (if not NULL)
// receives sum_i W_i = rho - rho0 without the FP32 cancellation of sums of
// values near w_i.
template <int Q, int FMT, bool PULL, bool WANT_F>
__device__ __forceinline__ void gather(const Launch &L, const Site &s, typename Fmt<FMT>::T *f,
                                       typename Fmt<FMT>::T *g, typename Fmt<FMT>::T *wsum = nullptr) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    constexpr bool DEV = Fmt<FMT>::DEV;
    const T rho0 = T(L.P.rho0);
    // U of this node's row; a pulled population comes from row y - c_iy
    const T U = DEV ? T(couette_u(L, s.y)) : T(0);
    const long long np = L.G.np;
    const int n = s.n;
    T ws = T(0);
    // f_i - w_i rho0 (16-bit formats) or f_i as stored
    auto ldW = [&](int i, int k, T Uk) -> T {
        if constexpr (DEV) return P::ldw(L.src, np, i, k, rho0, Uk);
        else return P::ldf(L.src, np, i, k, rho0, Uk);
    };
    // f_i from W_i (16-bit formats) or as stored
    auto ldf = [&](int i, int k, T Uk, T extra) {
        if constexpr (DEV) {
            const T W = P::ldw(L.src, np, i, k, rho0, Uk) + extra;
            ws += W;
            return W + T(Lat<Q>::w(i)) * rho0;
        } else {
            return P::ldf(L.src, np, i, k, rho0, Uk) + extra;
        }
    };
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (!PULL || i == 0) {
            if (WANT_F) f[i] = ldf(i, n, U, T(0));
            g[i] = P::ldg(L.src, np, i, n);
            continue;
        }
        T uwx = T(0), uwy = T(0);
        const int src = pull_source<Q, T>(L.G, s, i, uwx, uwy);
        if (src >= 0) {
            if (WANT_F) f[i] = ldf(i, src, DEV ? T(couette_u(L, s.y - Lat<Q>::cy(i))) : T(0), T(0));
            g[i] = P::ldg(L.src, np, i, src);
        } else {
            const int o = Lat<Q>::opp(i);
            const T cu = T(Lat<Q>::cx(i)) * uwx + T(Lat<Q>::cy(i)) * uwy;
            const T wi2 = T(2.0 * Lat<Q>::w(i) * 3.0);
            const T php = static_cast<const T *>(L.phi_prev)[n];
            if (L.G.interp) {
                // Four-roller, interpolated bounce-back (linear, Bouzidi,
                // Firdaouss and Lallemand 2001): the roller surface cuts the
                // link at x - q c_i.  q < 1/2: the opposite population
                // interpolated between x and x + c_i before it is reflected,
                // 2q f*_ibar(x) + (1 - 2q) f*_ibar(x + c_i) (half-way
                // bounce-back where x + c_i is solid too); q >= 1/2: the
                // reflected one interpolated with the node's own,
                // [f*_ibar(x) + (2q - 1) f*_i(x)] / (2q).  The moving-wall
                // term takes weight 1 and 1/(2q) respectively; c_i . u_w is
                // the same at every point of the link (the rotation's
                // c_i x (p - c_k) does not change along c_i).  The weights
                // of each rule sum to 1, so 16-bit deviations combine alike.
                // The crossing and the wall velocity, in FP64 and rounded
                // once to the format (the row kernels take both from a
                // table made at create; this per-node path serves small or
                // odd-sized lattices and first steps), measured from the
                // node's periodic image beside the roller (the wrapped
                // source plus c_i)
                const int k = L.G.solid[site_src<Q>(s, i)];
                const int cxi = Lat<Q>::cx(i), cyi = Lat<Q>::cy(i);
                const int xi = wrapi(s.x - cxi, L.G.nx) + cxi, yi = wrapi(s.y - cyi, L.G.ny) + cyi;
                const double ex = cxi, ey = cyi;
                const double dx = xi - L.G.rcx[k], dy = yi - L.G.rcy[k];
                const double cc = ex * ex + ey * ey, dc = dx * ex + dy * ey;
                const double dd = dx * dx + dy * dy - L.G.rr * L.G.rr;
                const double disc = dc * dc - cc * dd;
                // first crossing (dc - sqrt(disc)) / cc, written as
                // dd / (dc + sqrt(disc)): the roots' product dd/cc and sum
                // 2 dc/cc are positive, so no cancellation for small q
                double qd = dd / (dc + sqrt(disc > 0.0 ? disc : 0.0));
                qd = qd <= 0.0 ? 1e-12 : (qd > 1.0 ? 1.0 : qd);
                const T q2 = T(2.0 * qd);
                const T cuk = T(L.G.om[k] * (ey * dx - ex * dy));  // c_i . u_w on the link
                const T lf = wi2 * rho0 * cuk, lg = wi2 * php * cuk;
                const int nb = site_nb<Q>(s, i);
                T Wv, gv;
                if (qd < 0.5 && !L.G.solid[nb]) {
                    const T Unb = DEV ? T(couette_u(L, s.y + Lat<Q>::cy(i))) : T(0);
                    Wv = q2 * ldW(o, n, U) + (T(1) - q2) * ldW(o, nb, Unb) + lf;
                    gv = q2 * P::ldg(L.src, np, o, n) + (T(1) - q2) * P::ldg(L.src, np, o, nb) + lg;
                } else if (qd >= 0.5) {
                    Wv = (ldW(o, n, U) + (q2 - T(1)) * ldW(i, n, U) + lf) / q2;
                    gv = (P::ldg(L.src, np, o, n) + (q2 - T(1)) * P::ldg(L.src, np, i, n) + lg) / q2;
                } else {
                    Wv = ldW(o, n, U) + lf;
                    gv = P::ldg(L.src, np, o, n) + lg;
                }
                if (WANT_F) {
                    if constexpr (DEV) {
                        ws += Wv;
                        f[i] = Wv + T(Lat<Q>::w(i)) * rho0;
                    } else {
                        f[i] = Wv;
                    }
                }
                g[i] = gv;
                continue;
            }
            // w_opp(i) = w_i: the opposite's deviation carries over
            if (WANT_F) f[i] = ldf(o, n, U, wi2 * rho0 * cu);
            g[i] = P::ldg(L.src, np, o, n) + wi2 * php * cu;
        }
    }
    if (wsum) *wsum = ws;
}

// Macroscopic state of a node: moments, force and velocity (Algorithm 1
// up to the velocity).
template <typename T>
struct Macro {
    T rho, phi, mu, ux, uy, uz, Fx, Fy, Fz;
};

template <int Q, int FMT>
__device__ __forceinline__ Macro<typename Fmt<FMT>::T> macro_of(const Launch &L, const Site &s,
                                                                 const typename Fmt<FMT>::T *f,
                                                                 const typename Fmt<FMT>::T *g) {
    using T = typename Fmt<FMT>::T;
    Macro<T> m;
    T rho = T(0), ph = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        ph += g[i];
        if (Lat<Q>::cx(i)) jx += T(Lat<Q>::cx(i)) * f[i];
        if (Lat<Q>::cy(i)) jy += T(Lat<Q>::cy(i)) * f[i];
        if (Lat<Q>::cz(i)) jz += T(Lat<Q>::cz(i)) * f[i];
    }
    // F = -phi grad(mu) = mu grad(phi) - grad(phi mu), isotropic gradients
    const T *__restrict__ phif = static_cast<const T *>(L.phi);
    const T *__restrict__ muf = static_cast<const T *>(L.mu);
    T gpx = T(0), gpy = T(0), gpz = T(0), gqx = T(0), gqy = T(0), gqz = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int k = site_nb<Q>(s, i);
        const T p = phif[k];
        const T pm = p * muf[k];
        const T w = T(Lat<Q>::w(i));
        if (Lat<Q>::cx(i)) { gpx += w * T(Lat<Q>::cx(i)) * p; gqx += w * T(Lat<Q>::cx(i)) * pm; }
        if (Lat<Q>::cy(i)) { gpy += w * T(Lat<Q>::cy(i)) * p; gqy += w * T(Lat<Q>::cy(i)) * pm; }
        if (Lat<Q>::cz(i)) { gpz += w * T(Lat<Q>::cz(i)) * p; gqz += w * T(Lat<Q>::cz(i)) * pm; }
    }
    const T mu = muf[s.n];
    m.Fx = T(3) * (mu * gpx - gqx);
    m.Fy = T(3) * (mu * gpy - gqy);
    m.Fz = T(3) * (mu * gpz - gqz);
    if (L.P.model == 1) {
        // full functional: -rho grad(mu_rho) = mu_rho grad(rho) - grad(rho mu_rho)
        const T *__restrict__ rf = static_cast<const T *>(L.rhof);
        const T *__restrict__ mr = static_cast<const T *>(L.murho);
        T grx = T(0), gry = T(0), grz = T(0), gsx = T(0), gsy = T(0), gsz = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int k = site_nb<Q>(s, i);
            const T r = rf[k];
            const T rm = r * mr[k];
            const T w = T(Lat<Q>::w(i));
            if (Lat<Q>::cx(i)) { grx += w * T(Lat<Q>::cx(i)) * r; gsx += w * T(Lat<Q>::cx(i)) * rm; }
            if (Lat<Q>::cy(i)) { gry += w * T(Lat<Q>::cy(i)) * r; gsy += w * T(Lat<Q>::cy(i)) * rm; }
            if (Lat<Q>::cz(i)) { grz += w * T(Lat<Q>::cz(i)) * r; gsz += w * T(Lat<Q>::cz(i)) * rm; }
        }
        const T mur = mr[s.n];
        m.Fx += T(3) * (mur * grx - gsx);
        m.Fy += T(3) * (mur * gry - gsy);
        m.Fz += T(3) * (mur * grz - gsz);
    }
    const T inv = T(1) / rho;
    m.ux = (jx + T(0.5) * m.Fx) * inv;
    m.uy = (jy + T(0.5) * m.Fy) * inv;
    m.uz = (jz + T(0.5) * m.Fz) * inv;
    m.rho = rho;
    m.phi = ph;
    m.mu = mu;
    return m;
}

// ------------------------------------------------------------------ kernels
//
// Lattice kernels run on a 3D grid: a block of kBX x kBY threads covers kBX
// consecutive x and kBY consecutive y at one z.

constexpr int kBX = 64;
constexpr int kBY = 4;
static_assert(kBX * kBY == kBlock, "block shape");

#define FRE_SITE_OR_RETURN(L, s)                                        \
    const int x_ = blockIdx.x * kBX + (threadIdx.x & (kBX - 1));        \
    const int y_ = blockIdx.y * kBY + (threadIdx.x / kBX);              \
    const int z_ = blockIdx.z;                                          \
    if (x_ >= (L).G.nx || y_ >= (L).G.ny) return;                      \
    const Site s = make_site((L).G, x_, y_, z_)

// phi = sum of the pulled g at one node
// (the full functional, model 1, also writes rho = sum of the pulled f)
template <int Q, int FMT, bool PULL>
__device__ __forceinline__ void node_phi(const Launch &L, const Site &s) {
    using T = typename Fmt<FMT>::T;
    T g[Q];
    if (L.P.model == 1) {
        T f[Q];
        gather<Q, FMT, PULL, true>(L, s, f, g);
        T r = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) r += f[i];
        static_cast<T *>(L.rhof)[s.n] = r;
    } else {
        gather<Q, FMT, PULL, false>(L, s, nullptr, g);
    }
    T ph = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) ph += g[i];
    static_cast<T *>(L.phi)[s.n] = ph;
}

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_phi(Launch L) {
    pdl_wait();
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) return;
    node_phi<Q, FMT, PULL>(L, s);
}

// Stencil value at roller solid ghost[t]: w-weighted mean over fluid neighbours.
template <int Q, typename T>
__device__ __forceinline__ void node_ghost(const Launch &L, T *field, int t) {
    int x, y, z;
    decode(L.G, L.ghost[t], x, y, z);
    const Site s = make_site(L.G, x, y, z);
    T num = T(0), den = T(0);
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        const int m = site_nb<Q>(s, j);
        if (L.G.solid[m]) continue;
        num += T(Lat<Q>::w(j)) * field[m];
        den += T(Lat<Q>::w(j));
    }
    field[s.n] = den > T(0) ? num / den : T(0);
}

template <int Q, typename T>
__global__ void __launch_bounds__(kBlock) k_ghost(Launch L, T *field) {
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.n_ghost) return;
    node_ghost<Q, T>(L, field, t);
}

// mu = A (phi^3 - phi) - kappa lap(phi), lap = (2/cs^2) sum w_i (phi(x+c_i) - phi(x))
// Full functional (model 1, Eq. mu_rho and Eq. mu_phi), a = rho + phi,
// b = rho - phi:
//   mu_rho = k1/8 a(a-2)(a-1) + k2/8 b(b-2)(b-1)
//            + alpha^2/4 [-(k1 + k2) lap(rho) + (k2 - k1) lap(phi)],
//   mu_phi = k1/8 a(a-2)(a-1) - k2/8 b(b-2)(b-1)
//            + alpha^2/4 [-(k1 + k2) lap(phi) + (k2 - k1) lap(rho)];
// mu_phi goes to L.mu, mu_rho to L.murho.
template <int Q, typename T>
__device__ __forceinline__ void node_mu(const Launch &L, const Site &s) {
    const T *__restrict__ phi = static_cast<const T *>(L.phi);
    const T p0 = phi[s.n];
    T lap = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) lap += T(Lat<Q>::w(i)) * (phi[site_nb<Q>(s, i)] - p0);
    lap *= T(6);
    if (L.P.model == 1) {
        const T *__restrict__ rho = static_cast<const T *>(L.rhof);
        const T r0 = rho[s.n];
        T lapr = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) lapr += T(Lat<Q>::w(i)) * (rho[site_nb<Q>(s, i)] - r0);
        lapr *= T(6);
        const T k1 = T(L.P.kappa1), k2 = T(L.P.kappa2), al2 = T(L.P.alpha * L.P.alpha);
        const T a = r0 + p0, b = r0 - p0;
        const T ta = k1 / T(8) * a * (a - T(2)) * (a - T(1));
        const T tb = k2 / T(8) * b * (b - T(2)) * (b - T(1));
        static_cast<T *>(L.murho)[s.n] = ta + tb + al2 / T(4) * (-(k1 + k2) * lapr + (k2 - k1) * lap);
        static_cast<T *>(L.mu)[s.n] = ta - tb + al2 / T(4) * (-(k1 + k2) * lap + (k2 - k1) * lapr);
        return;
    }
    const T A = sizeof(T) == 4 ? T(L.F.A) : T(L.P.A), kappa = sizeof(T) == 4 ? T(L.F.kappa) : T(L.P.kappa);
    static_cast<T *>(L.mu)[s.n] = A * (p0 * p0 * p0 - p0) - kappa * lap;
}

template <int Q, typename T>
__global__ void __launch_bounds__(kBlock) k_mu(Launch L) {
    pdl_wait();
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) return;
    node_mu<Q, T>(L, s);
}

// Fused pull + collide of f and g for one node (Algorithm 1).
template <int Q, int FMT, bool PULL>
__device__ __forceinline__ void node_update(const Launch &L, const Site &s) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    const int n = s.n;
    T f[Q], g[Q];
    T wsum = T(0);  // 16-bit formats: rho - rho0 from the small deviations
    gather<Q, FMT, PULL, true>(L, s, f, g, &wsum);
    const Macro<T> m = macro_of<Q, FMT>(L, s, f, g);

    // FP32 computes take the constants rounded on the host
    const bool f32 = sizeof(T) == 4;
    const T of = f32 ? T(L.F.omega_f) : T(1.0 / L.P.tau_f), og = f32 ? T(L.F.omega_g) : T(1.0 / L.P.tau_g);
    const T kf = f32 ? T(L.F.kf) : T(1.0 - 0.5 / L.P.tau_f);
    const T gmu3 = (f32 ? T(L.F.gamma3) : T(3.0 * L.P.Gamma)) * m.mu;
    const T usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const T uF = m.ux * m.Fx + m.uy * m.Fy + m.uz * m.Fz;
    const T U = Fmt<FMT>::DEV ? T(couette_u(L, s.y)) : T(0);
    T fsum = T(0), gsum = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const T cx = T(Lat<Q>::cx(i)), cy = T(Lat<Q>::cy(i)), cz = T(Lat<Q>::cz(i));
        const T w = T(Lat<Q>::w(i));
        const T cu = cx * m.ux + cy * m.uy + cz * m.uz;
        const T cF = cx * m.Fx + cy * m.Fy + cz * m.Fz;
        const T poly = T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq;
        const T feq = w * m.rho * (T(1) + poly);
        // Guo: (1 - 1/2tau) w [3 (c - u).F + 9 (c.u)(c.F)]
        const T S = kf * w * (T(3) * (cF - uF) + T(9) * cu * cF);
        const T fs = f[i] - (f[i] - feq) * of + S;
        const T geq = w * (gmu3 + m.phi * poly);
        const T gs = g[i] - (g[i] - geq) * og;
        if constexpr (Fmt<FMT>::DEV)
            fsum += P::stw_back(L.dst, L.G.np, i, n, fs - T(Lat<Q>::w(i)) * T(L.P.rho0), T(L.P.rho0), U);
        else
            fsum += P::stf_back(L.dst, L.G.np, i, n, fs, T(L.P.rho0), U);
        gsum += P::stg_back(L.dst, L.G.np, i, n, gs);
        if (L.reflect) {
            // four-roller device run by the row kernels: when x + c_i is a
            // roller node, the next step pulls population opp(i) at x from
            // it; leave there f*_i(x) plus the moving-wall term of that link
            // (the row kernels read it as from any other source)
            const int nb = site_nb<Q>(s, i);
            const int k = L.G.solid[nb];
            if (k) {
                const int o = Lat<Q>::opp(i);
                // c_opp(i) . u_w = -(c_i . u_w), u_w = omega_k z x (x - c_k),
                // x in the frame of the roller (the wrapped roller node - c_i)
                const int xr = wrapi(s.x + Lat<Q>::cx(i), L.G.nx) - Lat<Q>::cx(i);
                const int yr = wrapi(s.y + Lat<Q>::cy(i), L.G.ny) - Lat<Q>::cy(i);
                const T cu = -T(L.G.om[k]) * (T(Lat<Q>::cy(i)) * (T(xr) - T(L.G.rcx[k])) -
                                               T(Lat<Q>::cx(i)) * (T(yr) - T(L.G.rcy[k])));
                const T wi6 = T(6.0 * Lat<Q>::w(i));
                P::stf(L.dst, L.G.np, o, nb, fs + wi6 * T(L.P.rho0) * cu, T(L.P.rho0), T(0));
                P::stg(L.dst, L.G.np, o, nb, gs + wi6 * m.phi * cu);
            }
        }
    }
    // rest populations close the collision invariants on the values as
    // stored: sum f* = rho, sum g* = phi (in the 16-bit formats up to the
    // rounding of the stored f*_0; g*_0 is FP32).  16-bit f closes on the
    // deviations from w_i rho0: (rho - rho0) - sum_{i>0} W*_i
    if constexpr (Fmt<FMT>::DEV)
        P::stw_back(L.dst, L.G.np, 0, n, wsum - fsum, T(L.P.rho0), U);
    else
        P::stf(L.dst, L.G.np, 0, n, m.rho - fsum, T(L.P.rho0), U);
    P::stg(L.dst, L.G.np, 0, n, m.phi - gsum);
}

// Four-roller device on the row kernels: the wall links of the step just
// taken, reflected ahead of the next one (half-way bounce-back with the
// moving-wall term).  For population i at a fluid node x whose source x - c_i
// is a roller node, the next step pulls slot i of that roller node; leave
// there f*_opp(i)(x) + c rho0 and g*_opp(i)(x) + c phi(x, t), with
// c = 2 w_i (c_i . u_w) / cs^2 from the link table.  One thread per link
// and z plane.  Reads touch fluid nodes only, each roller slot has a single
// writer.  16-bit f holds deviations from w_i rho0 on this device, and
// w_opp(i) = w_i, so a deviation carries over; 16-bit g keeps i >= 1 in
// plane i - 1 (a link has c_i != 0).
constexpr int kReflectPlanes = 4;
template <int FMT>
__global__ void __launch_bounds__(kBlock) k_reflect(Launch L) {
    static_assert(FMT != FRE_FP64, "the row kernels compute in FP32");
    using S = typename Fmt<FMT>::S;
    constexpr bool DEV = Fmt<FMT>::DEV;
    pdl_wait();
    // kReflectPlanes planes of one link per thread: the table entry is read
    // once and the loads of all planes are in flight together (the pass is
    // bound by the latency of its scattered reads)
    constexpr int PZ = kReflectPlanes;
    const int nl = L.G.n_rlinks, nz = L.G.nz;
    const int nzc = (nz + PZ - 1) / PZ;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nl * nzc) return;
    const int zc = (int)(t / nl);
    const int4 e = __ldg(L.G.rlinks + (t - (long long)zc * nl));
    const int i = e.z & 0xff, o = (e.z >> 8) & 0xff, cz = ((e.z >> 16) & 0xff) - 1;
    const float c = __int_as_float(e.w);
    const size_t plane = (size_t)L.G.nx * L.G.ny, np = (size_t)L.G.np;
    S *f = static_cast<S *>(L.dst.f);
    S *g = static_cast<S *>(L.dst.g);
    const float *phi = static_cast<const float *>(L.phi);
    // 16-bit g keeps population i >= 1 in plane i - 1
    const size_t gi = DEV ? (size_t)(i - 1) : (size_t)i, go = DEV ? (size_t)(o - 1) : (size_t)o;
    float ph[PZ], fo[PZ], gq[PZ];
#pragma unroll
    for (int q = 0; q < PZ; ++q) {
        const int z = zc * PZ + q;
        if (z < nz) {
            const size_t n = (size_t)z * plane + (size_t)e.x;
            ph[q] = phi[n];
            fo[q] = to_float(f[(size_t)o * np + n]);
            gq[q] = to_float(g[go * np + n]);
        }
    }
#pragma unroll
    for (int q = 0; q < PZ; ++q) {
        const int z = zc * PZ + q;
        if (z < nz) {
            const size_t src = (size_t)wrapi(z - cz, nz) * plane + (size_t)e.y;
            f[(size_t)i * np + src] = from_float<S>(fmaf(c, L.F.rho0, fo[q]));
            g[gi * np + src] = from_float<S>(fmaf(c, ph[q], gq[q]));
        }
    }
}

// Interpolated roller walls on the row kernels: the linear rule of
// Bouzidi, Firdaouss and Lallemand that gather applies per node, evaluated
// once per wall link after the update from the post-collision values of
// fluid nodes, and written into slot i of the link's roller source, which
// the next step pulls like any other.  With the link's fraction q and
// moving-wall coefficient c (the tables Geo::rlinkq and Geo::rlinks):
//   q < 1/2, x + c_i fluid:       2q f*_ibar(x) + (1 - 2q) f*_ibar(x + c_i) + c rho0
//   q < 1/2, x + c_i a roller node: f*_ibar(x) + c rho0
//   q >= 1/2:                     [f*_ibar(x) + (2q - 1) f*_i(x) + c rho0] / (2q)
// and g alike with c phi(x, t).  The weights of each rule sum to 1, so
// 16-bit f combines as deviations from w_i rho0 (w_ibar = w_i).  Reads
// touch fluid nodes only, each roller slot has a single writer.
template <int FMT>
__global__ void __launch_bounds__(kBlock) k_reflect_interp(Launch L) {
    static_assert(FMT != FRE_FP64, "the row kernels compute in FP32");
    using S = typename Fmt<FMT>::S;
    constexpr bool DEV = Fmt<FMT>::DEV;
    pdl_wait();
    constexpr int PZ = kReflectPlanes;
    const int nl = L.G.n_rlinks, nz = L.G.nz;
    const int nzc = (nz + PZ - 1) / PZ;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nl * nzc) return;
    const int zc = (int)(t / nl);
    const int l = (int)(t - (long long)zc * nl);
    const int4 e = __ldg(L.G.rlinks + l);
    const int4 a = __ldg(L.G.rlinkq + l);
    const int i = e.z & 0xff, o = (e.z >> 8) & 0xff, cz = ((e.z >> 16) & 0xff) - 1;
    const float c = __int_as_float(e.w);
    const float q2 = 2.f * __int_as_float(a.x);
    const bool near = q2 < 1.f, nb_solid = a.z != 0;
    const size_t plane = (size_t)L.G.nx * L.G.ny, np = (size_t)L.G.np;
    S *f = static_cast<S *>(L.dst.f);
    S *g = static_cast<S *>(L.dst.g);
    const float *phi = static_cast<const float *>(L.phi);
    const size_t gi = DEV ? (size_t)(i - 1) : (size_t)i, go = DEV ? (size_t)(o - 1) : (size_t)o;
    const float rho0 = L.F.rho0;
#pragma unroll
    for (int q = 0; q < PZ; ++q) {
        const int z = zc * PZ + q;
        if (z >= nz) break;
        const size_t n = (size_t)z * plane + (size_t)e.x;
        const float ph = phi[n];
        const float fo = to_float(f[(size_t)o * np + n]), gov = to_float(g[go * np + n]);
        float fv, gv;
        if (near) {
            if (nb_solid) {
                fv = fo + c * rho0;
                gv = gov + c * ph;
            } else {
                const size_t nb = (size_t)wrapi(z + cz, nz) * plane + (size_t)a.y;
                fv = q2 * fo + (1.f - q2) * to_float(f[(size_t)o * np + nb]) + c * rho0;
                gv = q2 * gov + (1.f - q2) * to_float(g[go * np + nb]) + c * ph;
            }
        } else {
            fv = (fo + (q2 - 1.f) * to_float(f[(size_t)i * np + n]) + c * rho0) / q2;
            gv = (gov + (q2 - 1.f) * to_float(g[gi * np + n]) + c * ph) / q2;
        }
        const size_t src = (size_t)wrapi(z - cz, nz) * plane + (size_t)e.y;
        f[(size_t)i * np + src] = from_float<S>(fv);
        g[gi * np + src] = from_float<S>(gv);
    }
}

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_update(Launch L) {
    pdl_wait();
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) return;
    node_update<Q, FMT, PULL>(L, s);
}
// The D3Q19 FP32 / 16-bit update held to four resident blocks per SM (64
// registers, some spilled): the per-node kernels are latency-bound, and on
// the four-roller lattices the extra warps outweigh the spills (192x96x96:
// FP32 211 -> 198 us, FP16 283 -> 226 us).  D2Q9 fits five blocks unbounded.
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock, 4) k_update4(Launch L) {
    pdl_wait();
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) return;
    node_update<Q, FMT, PULL>(L, s);
}

// Macroscopic fields -> staging (FP64): rho, ux, uy, uz, phi, mu.
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_macro(Launch L) {
    using T = typename Fmt<FMT>::T;
    FRE_SITE_OR_RETURN(L, s);
    double *out = L.staging;
    const long long N = L.G.n;
    const int n = s.n;
    if (is_solid(L.G, n)) {
        for (int k = 0; k < 6; ++k) out[k * N + n] = 0.0;
        return;
    }
    T f[Q], g[Q];
    gather<Q, FMT, PULL, true>(L, s, f, g);
    const Macro<T> m = macro_of<Q, FMT>(L, s, f, g);
    out[0 * N + n] = m.rho;
    out[1 * N + n] = m.ux;
    out[2 * N + n] = m.uy;
    out[3 * N + n] = m.uz;
    out[4 * N + n] = m.phi;
    out[5 * N + n] = m.mu;
}

// Pre-collision population i of f (lat_g = 0) or g (lat_g = 1) -> staging.
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_pull_plane(Launch L, int lat_g, int i) {
    using T = typename Fmt<FMT>::T;
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) {
        L.staging[s.n] = 0.0;
        return;
    }
    T f[Q], g[Q];
    gather<Q, FMT, PULL, true>(L, s, f, g);
    T v = T(0);
#pragma unroll
    for (int j = 0; j < Q; ++j)
        if (j == i) v = lat_g ? g[j] : f[j];
    L.staging[s.n] = (double)v;
}

// staging -> pre-collision population i of the source buffer.
template <int Q, int FMT>
__global__ void __launch_bounds__(kBlock) k_load_plane(Launch L, int lat_g, int i) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    FRE_SITE_OR_RETURN(L, s);
    const int n = s.n;
    const T v = is_solid(L.G, n) ? T(0) : T(L.staging[n]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        if (j != i) continue;
        if (lat_g) P::stg(L.src, L.G.np, j, n, v);
        else P::stf(L.src, L.G.np, j, n, v, T(L.P.rho0), T(couette_u(L, s.y)));
    }
}

// phi field: droplet tanh((R - |x - c|)/(sqrt(2) xi)) or staging field 4.
template <int Q, typename T>
__global__ void __launch_bounds__(kBlock) k_set_phi(Launch L, int analytic, double cx, double cy, double cz,
                                                    double R) {
    FRE_SITE_OR_RETURN(L, s);
    T *phi = static_cast<T *>(L.phi);
    if (is_solid(L.G, s.n)) {
        phi[s.n] = T(0);
        return;
    }
    if (L.P.model == 1)
        static_cast<T *>(L.rhof)[s.n] = analytic ? T(L.P.rho0) : T(L.staging[s.n]);
    if (!analytic) {
        phi[s.n] = T(L.staging[4 * L.G.n + s.n]);
        return;
    }
    double dx = s.x - cx, dy = s.y - cy, dz = (Lat<Q>::D == 3) ? s.z - cz : 0.0;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    // interface width: xi = sqrt(kappa / A); the full functional's planar
    // profile tanh(x / (2 alpha)) has xi = sqrt(2) alpha
    double xi = L.P.model == 1 ? sqrt(2.0) * L.P.alpha : sqrt(L.P.kappa / L.P.A);
    phi[s.n] = T(tanh((R - r) / (sqrt(2.0) * xi)));
}

// f = f_eq(rho, u), g = g_eq(phi, mu, u) into the source buffer.  rho, u
// from staging fields 0..3, or rho0 and the analytic initial velocity.
template <int Q, int FMT>
__global__ void __launch_bounds__(kBlock) k_init_eq(Launch L, int from_staging) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    FRE_SITE_OR_RETURN(L, s);
    const long long N = L.G.n;
    const int n = s.n;
    const T rho0 = T(L.P.rho0);
    const T U = T(couette_u(L, s.y));
    if (is_solid(L.G, n)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            P::stf(L.src, L.G.np, i, n, T(0), rho0, U);
            P::stg(L.src, L.G.np, i, n, T(0));
        }
        return;
    }
    T rho, ux, uy, uz;
    if (from_staging) {
        rho = T(L.staging[0 * N + n]);
        ux = T(L.staging[1 * N + n]);
        uy = T(L.staging[2 * N + n]);
        uz = T(L.staging[3 * N + n]);
    } else {
        rho = rho0;
        ux = (L.G.device == FRE_SHEAR) ? T(L.G.uwall * (2.0 * (s.y + 0.5) / L.G.ny - 1.0)) : T(0);
        uy = T(0);
        uz = T(0);
    }
    const T phi = static_cast<const T *>(L.phi)[n];
    const T mu = static_cast<const T *>(L.mu)[n];
    const T usq = ux * ux + uy * uy + uz * uz;
    T gsum = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = T(Lat<Q>::cx(i)) * ux + T(Lat<Q>::cy(i)) * uy + T(Lat<Q>::cz(i)) * uz;
        const T poly = T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq;
        const T w = T(Lat<Q>::w(i));
        P::stf(L.src, L.G.np, i, n, w * rho * (T(1) + poly), rho0, U);
        if (i > 0) {
            const T ge = w * (T(3.0 * L.P.Gamma) * mu + phi * poly);
            gsum += ge;
            P::stg(L.src, L.G.np, i, n, ge);
        }
    }
    P::stg(L.src, L.G.np, 0, n, phi - gsum);
}

// ------------------------------------------------ consistent initialisation
//
// Consistent initial populations (Sec. 2.3: equilibrium populations whose
// kinetic moments are aligned by collisions before the simulated time
// starts, after Mei et al.): with the velocity u0 and the force F0 of the
// initial state held fixed, f is collided (density free) and streamed
// `iterations` times; g ends at g_eq(phi0, mu0, u0).  Staging fields 0..2
// hold u0, 3..5 hold F0.

// u0 = sum c_i f_i / rho and F0 (from the current phi and mu fields) of
// the in-place state
template <int Q, int FMT>
__global__ void __launch_bounds__(kBlock) k_mei_prep(Launch L) {
    using T = typename Fmt<FMT>::T;
    FRE_SITE_OR_RETURN(L, s);
    const long long N = L.G.n;
    double *st = L.staging;
    if (is_solid(L.G, s.n)) {
        for (int k = 0; k < 6; ++k) st[k * N + s.n] = 0.0;
        return;
    }
    T f[Q], g[Q];
    gather<Q, FMT, false, true>(L, s, f, g);
    const Macro<T> m = macro_of<Q, FMT>(L, s, f, g);
    T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        jx += T(Lat<Q>::cx(i)) * f[i];
        jy += T(Lat<Q>::cy(i)) * f[i];
        jz += T(Lat<Q>::cz(i)) * f[i];
    }
    st[0 * N + s.n] = jx / m.rho;
    st[1 * N + s.n] = jy / m.rho;
    st[2 * N + s.n] = jz / m.rho;
    st[3 * N + s.n] = m.Fx;
    st[4 * N + s.n] = m.Fy;
    st[5 * N + s.n] = m.Fz;
}

// one pass: pull (or read in place) f, collide with u0 and F0 held, store
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_mei_iter(Launch L) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    FRE_SITE_OR_RETURN(L, s);
    if (is_solid(L.G, s.n)) return;
    const int n = s.n;
    const long long N = L.G.n;
    T f[Q], g[Q];
    T wsum = T(0);
    gather<Q, FMT, PULL, true>(L, s, f, g, &wsum);
    T rho = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) rho += f[i];
    const double *st = L.staging;
    const T ux = T(st[n]), uy = T(st[N + n]), uz = T(st[2 * N + n]);
    const T Fx = T(st[3 * N + n]), Fy = T(st[4 * N + n]), Fz = T(st[5 * N + n]);
    const bool f32 = sizeof(T) == 4;
    const T of = f32 ? T(L.F.omega_f) : T(1.0 / L.P.tau_f);
    const T kf = f32 ? T(L.F.kf) : T(1.0 - 0.5 / L.P.tau_f);
    const T rho0 = T(L.P.rho0);
    const T U = Fmt<FMT>::DEV ? T(couette_u(L, s.y)) : T(0);
    const T usq = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;
    T fsum = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const T cx = T(Lat<Q>::cx(i)), cy = T(Lat<Q>::cy(i)), cz = T(Lat<Q>::cz(i));
        const T w = T(Lat<Q>::w(i));
        const T cu = cx * ux + cy * uy + cz * uz;
        const T cF = cx * Fx + cy * Fy + cz * Fz;
        const T feq = w * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
        const T S = kf * w * (T(3) * (cF - uF) + T(9) * cu * cF);
        const T fs = f[i] - (f[i] - feq) * of + S;
        if constexpr (Fmt<FMT>::DEV)
            fsum += P::stw_back(L.dst, L.G.np, i, n, fs - w * rho0, rho0, U);
        else
            fsum += P::stf_back(L.dst, L.G.np, i, n, fs, rho0, U);
    }
    // the rest population closes the mass on the stored values
    if constexpr (Fmt<FMT>::DEV)
        P::stw_back(L.dst, L.G.np, 0, n, wsum - fsum, rho0, U);
    else
        P::stf(L.dst, L.G.np, 0, n, rho - fsum, rho0, U);
}

// the pre-collision state of step 0: the pulled f, and g = g_eq(phi0, mu0, u0)
template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_mei_final(Launch L) {
    using T = typename Fmt<FMT>::T;
    using P = Pop<Q, FMT>;
    FRE_SITE_OR_RETURN(L, s);
    const int n = s.n;
    const long long N = L.G.n;
    const T rho0 = T(L.P.rho0);
    const T U = Fmt<FMT>::DEV ? T(couette_u(L, s.y)) : T(0);
    if (is_solid(L.G, n)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            P::stf(L.dst, L.G.np, i, n, T(0), rho0, U);
            P::stg(L.dst, L.G.np, i, n, T(0));
        }
        return;
    }
    T f[Q], g[Q];
    gather<Q, FMT, PULL, true>(L, s, f, g);
#pragma unroll
    for (int i = 0; i < Q; ++i) P::stf(L.dst, L.G.np, i, n, f[i], rho0, U);
    const double *st = L.staging;
    const T ux = T(st[n]), uy = T(st[N + n]), uz = T(st[2 * N + n]);
    const T phi = static_cast<const T *>(L.phi)[n];
    const T mu = static_cast<const T *>(L.mu)[n];
    const T usq = ux * ux + uy * uy + uz * uz;
    const T gmu3 = T(3.0 * L.P.Gamma) * mu;
    T gsum = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const T cu = T(Lat<Q>::cx(i)) * ux + T(Lat<Q>::cy(i)) * uy + T(Lat<Q>::cz(i)) * uz;
        const T ge = T(Lat<Q>::w(i)) * (gmu3 + phi * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
        gsum += P::stg_back(L.dst, L.G.np, i, n, ge);
    }
    P::stg(L.dst, L.G.np, 0, n, phi - gsum);
}

// ------------------------------------------------------------ observables

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kObsVals = 10;   // rho, phi, vol, W, count, Wx, Wy, Wz, max|u|, non-finite
constexpr int kMomVals = 6;    // central second moments
constexpr int kRedBlocks = 1024;                      // max blocks of a reduction
constexpr int kRedMom = kRedBlocks * kObsVals;        // offset of pass-2 partials
constexpr int kRedTot = kRedBlocks * (kObsVals + kMomVals);  // offset of totals
constexpr int kRedDoubles = kRedTot + 32;             // size of the scratch

// Block reduction of NV values (sums except the two last, which are maxima
// when MAXLAST is set) into red[blockIdx.x * NV + k].
template <int NV, bool MAXLAST>
__device__ __forceinline__ void block_reduce_store(double *v, double *red) {
    __shared__ double sh[kBlock / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double r = (MAXLAST && k >= NV - 2) ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) sh[wid][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        double acc = sh[0][k];
        for (int w = 1; w < kBlock / 32; ++w) acc = (MAXLAST && k >= NV - 2) ? fmax(acc, sh[w][k]) : acc + sh[w][k];
        red[blockIdx.x * NV + k] = acc;
    }
}

template <int Q, int FMT, bool PULL>
__global__ void __launch_bounds__(kBlock) k_obs1(Launch L) {
    using T = typename Fmt<FMT>::T;
    double v[kObsVals];
#pragma unroll
    for (int k = 0; k < kObsVals; ++k) v[k] = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L.G.n; n += gridDim.x * blockDim.x) {
        if (is_solid(L.G, n)) continue;
        int x, y, z;
        decode(L.G, n, x, y, z);
        const Site s = make_site(L.G, x, y, z);
        T f[Q], g[Q];
        gather<Q, FMT, PULL, true>(L, s, f, g);
        const Macro<T> m = macro_of<Q, FMT>(L, s, f, g);
        const double rho = m.rho, ph = m.phi;
        const double u = sqrt((double)m.ux * m.ux + (double)m.uy * m.uy + (double)m.uz * m.uz);
        v[0] += rho;
        v[1] += ph;
        v[2] += 0.5 * (1.0 + ph);
        if (ph > 0.0) {
            const double w = 0.5 * (1.0 + ph);
            v[3] += w;
            v[4] += 1.0;
            v[5] += w * x;
            v[6] += w * y;
            v[7] += w * z;
        }
        if (isfinite(rho) && isfinite(ph) && isfinite(u) && isfinite((double)m.mu)) {
            v[8] = fmax(v[8], u);
        } else {
            v[9] = 1.0;
        }
    }
    block_reduce_store<kObsVals, true>(v, L.red);
}

// Sum the per-block partials in a fixed order (deterministic).
template <int NV, bool MAXLAST>
__global__ void k_reduce_partials(const double *red, int nblocks, double *out) {
    const int k = threadIdx.x;
    if (k >= NV) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        double x = red[b * NV + k];
        acc = (MAXLAST && k >= NV - 2) ? fmax(acc, x) : acc + x;
    }
    out[k] = acc;
}

template <int Q, typename T>
__global__ void __launch_bounds__(kBlock) k_obs2(Launch L, const double *tot) {
    double v[kMomVals];
#pragma unroll
    for (int k = 0; k < kMomVals; ++k) v[k] = 0.0;
    const double W = tot[3];
    const double X = W > 0 ? tot[5] / W : 0.0, Y = W > 0 ? tot[6] / W : 0.0, Z = W > 0 ? tot[7] / W : 0.0;
    const T *phi = static_cast<const T *>(L.phi);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L.G.n; n += gridDim.x * blockDim.x) {
        if (is_solid(L.G, n)) continue;
        const double ph = phi[n];
        if (!(ph > 0.0)) continue;
        int x, y, z;
        decode(L.G, n, x, y, z);
        const double w = 0.5 * (1.0 + ph);
        const double dx = x - X, dy = y - Y, dz = z - Z;
        v[0] += w * dx * dx;
        v[1] += w * dy * dy;
        v[2] += w * dz * dz;
        v[3] += w * dx * dy;
        v[4] += w * dx * dz;
        v[5] += w * dy * dz;
    }
    block_reduce_store<kMomVals, false>(v, L.red + kRedMom);
}

// Pressure at a node: cs^2 rho + phi mu - (A/4)(phi^2 - 1)^2.
template <int Q, int FMT, bool PULL>
__device__ double pressure_at(const Launch &L, int x, int y, int z) {
    using T = typename Fmt<FMT>::T;
    const Site s = make_site(L.G, x, y, z);
    T f[Q], g[Q];
    gather<Q, FMT, PULL, true>(L, s, f, g);
    double rho = 0.0;
    for (int i = 0; i < Q; ++i) rho += (double)f[i];
    const double ph = static_cast<const T *>(L.phi)[s.n];
    const double mu = static_cast<const T *>(L.mu)[s.n];
    if (L.P.model == 1) {
        // cs^2 rho + rho mu_rho + phi mu_phi - psi, psi the bulk part of
        // Eq. functional: k1/32 a^2 (a-2)^2 + k2/32 b^2 (b-2)^2
        const double mur = static_cast<const T *>(L.murho)[s.n];
        const double a = rho + ph, b = rho - ph;
        const double psi = L.P.kappa1 / 32.0 * a * a * (a - 2.0) * (a - 2.0) +
                           L.P.kappa2 / 32.0 * b * b * (b - 2.0) * (b - 2.0);
        return rho / 3.0 + rho * mur + ph * mu - psi;
    }
    return rho / 3.0 + ph * mu - 0.25 * L.P.A * (ph * ph - 1.0) * (ph * ph - 1.0);
}

// Pressure at the point (X, Y, Z) by trilinear interpolation of the nodal
// pressure: periodic in x and z, and in y off the shear device (whose y is
// clamped to the fluid rows); solid nodes carry no weight.  A droplet
// centred on a cell face would switch nodes under any rounding of its
// centroid if the pressure were read at the nearest node.
template <int Q, int FMT, bool PULL>
__device__ double pressure_interp(const Launch &L, double X, double Y, double Z) {
    const Geo &G = L.G;
    const int x0 = (int)floor(X), y0 = (int)floor(Y), z0 = (int)floor(Z);
    const double fx = X - x0, fy = Y - y0, fz = Z - z0;
    double acc = 0.0, wsum = 0.0;
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
        if (w == 0.0) continue;
        const int x = wrapi(x0 + dx, G.nx), z = wrapi(z0 + dz, G.nz);
        int y = y0 + dy;
        y = G.device == FRE_SHEAR ? (y < 0 ? 0 : (y >= G.ny ? G.ny - 1 : y)) : wrapi(y, G.ny);
        if (is_solid(G, node_index(G, x, y, z))) continue;
        acc += w * pressure_at<Q, FMT, PULL>(L, x, y, z);
        wsum += w;
    }
    return wsum > 0.0 ? acc / wsum : 0.0;
}

template <int Q, int FMT, bool PULL>
__global__ void k_obs_final(Launch L, const double *t1, const double *t2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fre_obs *o = L.obs;
    o->mass = t1[0];
    o->phi_sum = t1[1];
    o->volume = t1[2];
    o->drop_weight = t1[3];
    o->drop_count = t1[4];
    o->max_u = t1[8];
    const int bad = t1[9] != 0.0;
    const double W = t1[3];
    for (int k = 0; k < 3; ++k) o->centroid[k] = 0.0;
    for (int k = 0; k < 6; ++k) o->I[k] = 0.0;
    o->D = o->theta_deg = o->p_centre = o->p_far = o->dp = 0.0;
    if (W > 0.0) {
        const double X[3] = {t1[5] / W, t1[6] / W, t1[7] / W};
        for (int k = 0; k < 3; ++k) o->centroid[k] = X[k];
        for (int k = 0; k < 6; ++k) o->I[k] = t2[k] / W;
        const double a = o->I[0], b = o->I[1], c = o->I[3];
        const double mm = 0.5 * (a + b), r = sqrt(0.25 * (a - b) * (a - b) + c * c);
        double l1 = mm + r, l2 = mm - r;
        if (l2 < 0.0) l2 = 0.0;
        const double s1 = sqrt(l1), s2 = sqrt(l2);
        o->D = (s1 + s2) > 0.0 ? (s1 - s2) / (s1 + s2) : 0.0;
        o->theta_deg = 0.5 * atan2(2.0 * c, a - b) * (180.0 / 3.14159265358979323846);
        // Laplace pressure (Sec. 3): at the centroid vs half a period away
        // in x (and z)
        const Geo &G = L.G;
        o->p_centre = pressure_interp<Q, FMT, PULL>(L, X[0], X[1], X[2]);
        o->p_far = pressure_interp<Q, FMT, PULL>(L, X[0] + G.nx / 2, X[1], G.nz > 1 ? X[2] + G.nz / 2 : X[2]);
        o->dp = o->p_centre - o->p_far;
    }
    o->status = bad ? 1 : (o->max_u > 0.3 ? 2 : 0);
}

// ------------------------------------------------------------ launchers

inline unsigned grid_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }
inline dim3 grid3(const Geo &G) {
    return dim3((unsigned)((G.nx + kBX - 1) / kBX), (unsigned)((G.ny + kBY - 1) / kBY), (unsigned)G.nz);
}

template <int Q, int FMT>
struct Launchers {
    using T = typename Fmt<FMT>::T;

    static void phi(const Launch &L, bool pull) {
        if (pull) launch_pdl(k_phi<Q, FMT, true>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
        else launch_pdl(k_phi<Q, FMT, false>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
    }
    static void ghost(const Launch &L, void *field) {
        if (L.n_ghost > 0)
            launch_pdl(k_ghost<Q, T>, dim3(grid_for(L.n_ghost)), dim3(kBlock), 0, L.stream, L, static_cast<T *>(field));
    }
    static void mu(const Launch &L) { launch_pdl(k_mu<Q, T>, grid3(L.G), dim3(kBlock), 0, L.stream, L); }
    static void update(const Launch &L, bool pull) {
        if constexpr (Q == 19 && FMT != FRE_FP64) {
            if (pull) launch_pdl(k_update4<Q, FMT, true>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
            else launch_pdl(k_update4<Q, FMT, false>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
            return;
        }
        if (pull) launch_pdl(k_update<Q, FMT, true>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
        else launch_pdl(k_update<Q, FMT, false>, grid3(L.G), dim3(kBlock), 0, L.stream, L);
    }
    static void obs(const Launch &L, bool pull) {
        const int nb = L.red_blocks;
        double *t1 = L.red + kRedTot;
        double *t2 = t1 + 16;
        if (pull) k_obs1<Q, FMT, true><<<nb, kBlock, 0, L.stream>>>(L);
        else k_obs1<Q, FMT, false><<<nb, kBlock, 0, L.stream>>>(L);
        k_reduce_partials<kObsVals, true><<<1, 32, 0, L.stream>>>(L.red, nb, t1);
        k_obs2<Q, T><<<nb, kBlock, 0, L.stream>>>(L, t1);
        k_reduce_partials<kMomVals, false><<<1, 32, 0, L.stream>>>(L.red + kRedMom, nb, t2);
        if (pull) k_obs_final<Q, FMT, true><<<1, 32, 0, L.stream>>>(L, t1, t2);
        else k_obs_final<Q, FMT, false><<<1, 32, 0, L.stream>>>(L, t1, t2);
    }
    static void macro(const Launch &L, bool pull) {
        if (pull) k_macro<Q, FMT, true><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
        else k_macro<Q, FMT, false><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
    }
    static void pull_plane(const Launch &L, bool pull, int lat_g, int i) {
        if (pull) k_pull_plane<Q, FMT, true><<<grid3(L.G), kBlock, 0, L.stream>>>(L, lat_g, i);
        else k_pull_plane<Q, FMT, false><<<grid3(L.G), kBlock, 0, L.stream>>>(L, lat_g, i);
    }
    static void load_plane(const Launch &L, int lat_g, int i) {
        k_load_plane<Q, FMT><<<grid3(L.G), kBlock, 0, L.stream>>>(L, lat_g, i);
    }
    static void set_phi(const Launch &L, int analytic, double cx, double cy, double cz, double R) {
        k_set_phi<Q, T><<<grid3(L.G), kBlock, 0, L.stream>>>(L, analytic, cx, cy, cz, R);
    }
    static void init_eq(const Launch &L, int from_staging) {
        k_init_eq<Q, FMT><<<grid3(L.G), kBlock, 0, L.stream>>>(L, from_staging);
    }
    static void reflect(const Launch &L) {
        if constexpr (FMT != FRE_FP64) {
            const long long nt = (long long)L.G.n_rlinks * ((L.G.nz + kReflectPlanes - 1) / kReflectPlanes);
            if (nt > 0)
                launch_pdl(L.G.rlinkq ? k_reflect_interp<FMT> : k_reflect<FMT>,
                           dim3((unsigned)((nt + kBlock - 1) / kBlock)), dim3(kBlock), 0, L.stream, L);
        }
    }
    static void mei_prep(const Launch &L) { k_mei_prep<Q, FMT><<<grid3(L.G), kBlock, 0, L.stream>>>(L); }
    static void mei_iter(const Launch &L, bool pull) {
        if (pull) k_mei_iter<Q, FMT, true><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
        else k_mei_iter<Q, FMT, false><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
    }
    static void mei_final(const Launch &L, bool pull) {
        if (pull) k_mei_final<Q, FMT, true><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
        else k_mei_final<Q, FMT, false><<<grid3(L.G), kBlock, 0, L.stream>>>(L);
    }
};

}  // namespace fre
