// Host runtime of the C ABI declared in include/fre.h: validation, device
// memory, geometry, and the launch sequence of one time step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fre_ctx.h"

namespace fre {
// scratch layout of the observables reduction (see fre_kernels.cuh)
constexpr int kRedDoublesHost = 1024 * 16 + 32;
}  // namespace fre

namespace {

thread_local std::string g_err;

fre_status fail(fre_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define FRE_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(FRE_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Four-roller geometry (Sec. 3): four cylinders of radius nx/8 along z,
// centred at ((nx-1)/2 +- nx/4, (ny-1)/2 +- ny/4), top right and bottom left
// turning counter-clockwise, the other two clockwise, at surface speed
// u_wall; a node belongs to the first roller whose disc holds it.  One z
// plane of roller ids (the rollers are extruded along z).
struct RollerPlane {
    double rcx[5], rcy[5], om[5];
    std::vector<unsigned char> id;  // [ny][nx], 0 fluid
};

void roller_plane(const fre_params &p, RollerPlane &g) {
    const double cx = 0.5 * (p.nx - 1), cy = 0.5 * (p.ny - 1);
    const double ox = 0.25 * p.nx, oy = 0.25 * p.ny;
    const double r = p.nx / 8.0;
    const double om = p.u_wall / r;
    const double xs[5] = {0, cx + ox, cx - ox, cx - ox, cx + ox};
    const double ys[5] = {0, cy + oy, cy + oy, cy - oy, cy - oy};
    const double ws[5] = {0, om, -om, om, -om};  // top right, top left, bottom left, bottom right
    for (int k = 0; k < 5; ++k) {
        g.rcx[k] = xs[k];
        g.rcy[k] = ys[k];
        g.om[k] = ws[k];
    }
    g.id.assign((size_t)p.nx * p.ny, 0);
    for (int y = 0; y < p.ny; ++y)
        for (int x = 0; x < p.nx; ++x)
            for (int k = 1; k <= 4; ++k) {
                const double dx = x - xs[k], dy = y - ys[k];
                if (dx * dx + dy * dy <= r * r) {
                    g.id[(size_t)y * p.nx + x] = (unsigned char)k;
                    break;
                }
            }
}

const int kC9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                       {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
const int kC19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                         {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},
                         {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0}, {-1, 1, 0},
                         {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};

int wrap_host(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// The wall links of one plane: population i at fluid node (x, y) whose
// source (x, y) - c_i is a roller node of roller k, as the table of
// k_reflect (Geo::rlinks), ordered by i, then y, then x, so that the
// neighbouring threads of a warp read and write the same population plane
// at neighbouring boundary nodes (shared sectors where the boundary runs
// along x).  The moving-wall coefficient is
// 2 w_i (c_i . u_w) / cs^2 with u_w = omega_k z x (p - c_k) at the link's
// wall point p = x - c_i / 2; the shift along c_i drops out of c_i x (p - c_k),
// so c_i . u_w = omega_k (c_iy (x - x_k) - c_ix (y - y_k)), with (x, y) the
// node's image beside the roller (the wrapped source plus c_i: the rollers
// of boxes with ny = nx/2 reach across the periodic y boundary).  Returns the
// number of links; fills `out` when it is not NULL, and `outq` (the
// interpolated walls' entries of Geo::rlinkq) when it is not NULL.  The
// link from x toward x - c_i meets the circle of radius r about c_k at
// x - q c_i with q the smaller root of |d - q c|^2 = r^2 (d = x - c_k, the
// in-plane part of c_i): q = dd / (dc + sqrt(dc^2 - cc dd)), dc = d.c,
// cc = c.c, dd = d.d - r^2 (both roots positive, no cancellation).
long long roller_links(const fre_params &p, int q, const RollerPlane &g, std::vector<int4> *out,
                       std::vector<int4> *outq = nullptr) {
    if (out) out->clear();
    if (outq) outq->clear();
    long long count = 0;
    for (int i = 1; i < q; ++i)
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                if (g.id[(size_t)y * p.nx + x]) continue;
                const int *ci = q == 9 ? kC9[i] : kC19[i];
                const int xs = wrap_host(x - ci[0], p.nx), ys = wrap_host(y - ci[1], p.ny);
                const int k = g.id[(size_t)ys * p.nx + xs];
                if (!k) continue;
                ++count;
                if (!out) continue;
                int o = 0;
                for (int j = 0; j < q; ++j) {
                    const int *cj = q == 9 ? kC9[j] : kC19[j];
                    if (cj[0] == -ci[0] && cj[1] == -ci[1] && cj[2] == -ci[2]) o = j;
                }
                const int c2 = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
                const double w = q == 9 ? (c2 == 1 ? 1.0 / 9 : 1.0 / 36) : (c2 == 1 ? 1.0 / 18 : 1.0 / 36);
                // in the frame of the roller: the node's image beside it (the
                // wrapped source plus c_i)
                const double dx = xs + ci[0] - g.rcx[k], dy = ys + ci[1] - g.rcy[k];
                const double cu = g.om[k] * (ci[1] * dx - ci[0] * dy);
                const float coef = float(6.0 * w * cu);
                int4 e;
                e.x = y * p.nx + x;
                e.y = ys * p.nx + xs;
                e.z = i | (o << 8) | ((ci[2] + 1) << 16);
                std::memcpy(&e.w, &coef, sizeof(float));
                out->push_back(e);
                if (outq) {
                    // from the node's periodic image beside the roller (dx, dy)
                    const double r = p.nx / 8.0;
                    const double cc = ci[0] * ci[0] + ci[1] * ci[1], dc = dx * ci[0] + dy * ci[1];
                    const double dd = dx * dx + dy * dy - r * r, disc = dc * dc - cc * dd;
                    double t = dd / (dc + std::sqrt(disc > 0.0 ? disc : 0.0));
                    t = t <= 0.0 ? 1e-12 : (t > 1.0 ? 1.0 : t);
                    const float qf = float(t);
                    const int xn = wrap_host(x + ci[0], p.nx), yn = wrap_host(y + ci[1], p.ny);
                    int4 a;
                    std::memcpy(&a.x, &qf, sizeof(float));
                    a.y = yn * p.nx + xn;
                    a.z = g.id[(size_t)yn * p.nx + xn] ? 1 : 0;
                    a.w = 0;
                    outq->push_back(a);
                }
            }
    return count;
}

struct Sizes {
    int q, sz_store, sz_comp;
    long long n, np;
    size_t buf_bytes, field_bytes, solid_bytes;
    int model;  // 1: two more fields (rho, mu_rho)
};

bool sizes_of(const fre_params *p, Sizes &s, std::string *why) {
    auto bad = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (!p) return bad("params is NULL");
    if (p->lattice != FRE_D2Q9 && p->lattice != FRE_D3Q19) return bad("unknown lattice");
    if (p->precision < FRE_FP64 || p->precision > FRE_BF16DEV) return bad("unknown precision");
    if (p->device < FRE_SHEAR || p->device > FRE_PERIODIC) return bad("unknown device");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bad("lattice sizes must be >= 1");
    if (p->lattice == FRE_D2Q9 && p->nz != 1) return bad("D2Q9 needs nz = 1");
    if ((p->flags & FRE_FLAG_COUETTE_REFERENCE) && (p->flags & FRE_FLAG_REST_REFERENCE))
        return bad("FRE_FLAG_COUETTE_REFERENCE and FRE_FLAG_REST_REFERENCE exclude each other");
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return bad("tau_f and tau_g must be > 1/2");
    if (!(p->A >= 0.0) || !(p->kappa >= 0.0)) return bad("A and kappa must be >= 0");
    if (!std::isfinite(p->gamma_mob) || !std::isfinite(p->u_wall) || !(p->rho0 > 0.0))
        return bad("gamma_mob and u_wall must be finite, rho0 > 0");
    if (p->model != 0 && p->model != 1) return bad("unknown free-energy model (0 or 1)");
    if (p->model == 1 && !(p->kappa1 >= 0.0 && p->kappa2 >= 0.0 && p->alpha >= 0.0 && std::isfinite(p->kappa1) &&
                           std::isfinite(p->kappa2) && std::isfinite(p->alpha)))
        return bad("model 1 needs finite kappa1, kappa2, alpha >= 0");
    if (p->device == FRE_FOUR_ROLLER && (p->nx < 8 || p->ny < 8)) return bad("four-roller needs nx, ny >= 8");
    if ((p->flags & FRE_FLAG_INTERPOLATED_WALLS) && p->device != FRE_FOUR_ROLLER)
        return bad("FRE_FLAG_INTERPOLATED_WALLS applies to the four-roller device only");
    long long n = (long long)p->nx * p->ny * p->nz;
    if (n > (1LL << 30)) return bad("too many nodes (limit 2^30)");
    s.q = p->lattice == FRE_D2Q9 ? 9 : 19;
    s.n = n;
    // plane stride: a multiple of 64 elements (aligned rows for vector
    // access) with an odd number of 64-element blocks, so the q planes of a
    // population array never sit a large power of two apart (DRAM channel
    // aliasing of the q loads a thread issues)
    s.np = (n + 63) / 64 * 64;
    if ((s.np / 64) % 2 == 0) s.np += 64;
    s.sz_store = p->precision == FRE_FP64 ? 8 : (p->precision == FRE_FP32 ? 4 : 2);
    s.sz_comp = p->precision == FRE_FP64 ? 8 : 4;
    size_t plane = (size_t)s.np * s.sz_store;
    if (p->precision == FRE_FP64 || p->precision == FRE_FP32) {
        s.buf_bytes = 2 * (size_t)s.q * plane;
    } else {
        s.buf_bytes = (size_t)s.q * plane + (size_t)(s.q - 1) * plane + (size_t)s.np * 4;
    }
    s.field_bytes = (size_t)s.np * s.sz_comp;
    s.solid_bytes = 0;
    if (p->device == FRE_FOUR_ROLLER) {
        RollerPlane g;
        roller_plane(*p, g);
        const size_t nl = (size_t)roller_links(*p, s.q, g, nullptr);
        s.solid_bytes = (size_t)s.np + sizeof(int4) * nl * ((p->flags & FRE_FLAG_INTERPOLATED_WALLS) ? 2 : 1);
    }
    s.model = p->model;
    return true;
}

// roots the component labelling lists at most (fre_components)
constexpr int kCclCap = 4096;

// device bytes of the component labelling: labels and sizes per node, the
// root list (allocated on first use, counted in the budget from the start)
size_t ccl_bytes(const Sizes &s) { return 2 * sizeof(int) * (size_t)s.n + 16 * (size_t)kCclCap + 256; }

size_t total_bytes(const Sizes &s) {
    return 2 * s.buf_bytes + (3 + 2 * s.model) * s.field_bytes + s.solid_bytes +
           sizeof(double) * fre::kRedDoublesHost + sizeof(fre_obs) + ccl_bytes(s);
}

fre_status dev_alloc(fre_ctx *c, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return FRE_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(FRE_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(*ptr);
    e = cudaMemsetAsync(*ptr, 0, bytes, c->stream);
    if (e != cudaSuccess) return fail(FRE_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return FRE_OK;
}

// Four-roller geometry of a context: roller id of every node, the solid
// nodes that have a fluid stencil neighbour, and the wall links of a plane.
void build_rollers(fre_ctx *c, std::vector<unsigned char> &solid, std::vector<int> &ghost,
                   std::vector<int4> &links, std::vector<int4> &linkq) {
    const fre_params &p = c->p;
    fre::Geo &G = c->G;
    RollerPlane g;
    roller_plane(p, g);
    for (int k = 0; k < 5; ++k) {
        G.rcx[k] = g.rcx[k];
        G.rcy[k] = g.rcy[k];
        G.om[k] = g.om[k];
    }
    G.rr = p.nx / 8.0;
    G.interp = (p.flags & FRE_FLAG_INTERPOLATED_WALLS) ? 1 : 0;
    const size_t plane = (size_t)p.nx * p.ny;
    solid.resize((size_t)G.n);
    for (int z = 0; z < p.nz; ++z) std::memcpy(solid.data() + (size_t)z * plane, g.id.data(), plane);
    const int q = c->q;
    const auto &c9 = kC9;
    const auto &c19 = kC19;
    auto wrap = wrap_host;
    roller_links(p, q, g, &links, G.interp ? &linkq : nullptr);
    ghost.clear();
    for (int z = 0; z < p.nz; ++z)
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                size_t n = ((size_t)z * p.ny + y) * p.nx + x;
                if (!solid[n]) continue;
                for (int j = 1; j < q; ++j) {
                    const int *cj = q == 9 ? c9[j] : c19[j];
                    size_t m = ((size_t)wrap(z + cj[2], p.nz) * p.ny + wrap(y + cj[1], p.ny)) * p.nx +
                               wrap(x + cj[0], p.nx);
                    if (!solid[m]) {
                        ghost.push_back((int)n);
                        break;
                    }
                }
            }
}

}  // namespace

fre::Launch fre::ctx_launch(fre_ctx *c) {
    fre::Launch L{};
    L.G = c->G;
    L.P = c->P;
    const double tf = c->P.tau_f, tg = c->P.tau_g;
    // reference profile of the 16-bit f stores: the Couette profile of the
    // shear device unless FRE_FLAG_REST_REFERENCE
    const bool shear = c->G.device == FRE_SHEAR && !(c->p.flags & FRE_FLAG_REST_REFERENCE) &&
                       (c->p.precision == FRE_FP16DEV || c->p.precision == FRE_BF16DEV);
    L.F = {float(1.0 / tf), float(1.0 / tg), float(1.0 - 0.5 / tf), float(3.0 * c->P.Gamma),
           float(c->P.A), float(c->P.kappa), float(c->P.rho0), float(c->G.uwall),
           shear ? float(c->G.uwall * (1.0 / c->G.ny - 1.0)) : 0.f, shear ? float(2.0 * c->G.uwall / c->G.ny) : 0.f,
           {}, {}, {}};
    for (int k = 0; k < 5; ++k) {
        L.F.rcx[k] = float(c->G.rcx[k]);
        L.F.rcy[k] = float(c->G.rcy[k]);
        L.F.rom[k] = float(c->G.om[k]);
    }
    L.src = c->buf[c->cur];
    L.dst = c->buf[1 - c->cur];
    L.phi_prev = c->phi[c->pp];
    L.phi = c->phi[1 - c->pp];
    L.mu = c->mu;
    L.rhof = c->rhof;
    L.murho = c->murho;
    L.ghost = c->ghost;
    L.n_ghost = c->n_ghost;
    L.red = c->red;
    L.red_blocks = c->red_blocks;
    L.obs = c->obs_dev;
    L.staging = c->staging;
    L.stream = c->stream;
    L.W = c->row_w;
    L.err = c->err_dev;
    L.stall = (c->p.flags & FRE_FLAG_TEST_PIPELINE_STALL) ? 1 : 0;
    // the per-node update reflects half-way wall links itself where the row
    // kernels run the context; interpolated links are left to the
    // reflection pass, which follows every update then
    L.reflect = (c->fullrow && c->G.device == FRE_FOUR_ROLLER && !c->G.interp) ? 1 : 0;
    L.wait_ns = L.stall ? 5000000ull : 2000000000ull;
    return L;
}

// Issue the kernels of one time step on the context stream and advance the
// host-side state (buffer parity, step counter).
void fre::ctx_launch_step(fre_ctx *c) {
    fre::Launch L = ctx_launch(c);
    const bool pull = !c->local;
    // the four-roller device takes its in-place first step on the per-node
    // kernels (which reflect their wall links themselves); its pulled row
    // update leaves the wall links to the reflection pass
    const bool roll = c->G.device == FRE_FOUR_ROLLER;
    if (c->fullrow && (pull || !roll)) {
        c->ks->phi_fullrow(L, pull);
        if (c->n_ghost) c->ks->ghost(L, L.phi);
        c->ks->mu_fullrow(L);
        if (c->n_ghost) c->ks->ghost(L, L.mu);
        c->ks->update_fullrow(L, pull);
        if (roll) c->ks->reflect(L);
    } else if (c->rows) {
        c->ks->phi_rows(L, pull);
        c->ks->mu_rows(L);
        c->ks->update_rows(L, pull);
    } else {
        c->ks->phi(L, pull);
        if (c->n_ghost) fre::ghost_fields(c, L, false);
        c->ks->mu(L);
        if (c->n_ghost) fre::ghost_fields(c, L, true);
        c->ks->update(L, pull);
        // the in-place step of interpolated walls on the row kernels: the
        // next (pulled, row) step reads its wall links from the roller slots
        if (c->fullrow && roll && c->G.interp) c->ks->reflect(L);
    }
    c->cur ^= 1;
    c->pp ^= 1;
    c->local = false;
    c->step++;
}

// Stencil values at the roller solids: phi (and rho, model 1) after the phi
// pass, mu (and mu_rho) after the mu pass.
void fre::ghost_fields(fre_ctx *c, const Launch &L, bool mu_pass) {
    c->ks->ghost(L, mu_pass ? L.mu : L.phi);
    if (c->P.model == 1) c->ks->ghost(L, mu_pass ? L.murho : L.rhof);
}

bool fre::same_geometry(const fre_params *p, const fre_params *q) {
    return p->lattice == q->lattice && p->precision == q->precision && p->device == q->device && p->nx == q->nx &&
           p->ny == q->ny && p->nz == q->nz && p->flags == q->flags && p->model == q->model;
}

fre_status fre::ctx_reparam(fre_ctx *c, const fre_params *p) {
    if (!c || !p) return fail(FRE_ERR_ARG, "ctx_reparam: NULL argument");
    if (!same_geometry(&c->p, p)) return fail(FRE_ERR_ARG, "ctx_reparam: geometry differs");
    Sizes s;
    std::string why;
    if (!sizes_of(p, s, &why)) return fail(FRE_ERR_ARG, "ctx_reparam: %s", why.c_str());
    c->p = *p;
    c->G.uwall = p->u_wall;
    c->P = {p->tau_f, p->tau_g, p->A, p->kappa, p->gamma_mob, p->rho0, p->model, p->kappa1, p->kappa2, p->alpha};
    c->initialised = false;
    return FRE_OK;
}

namespace {

fre::Launch launch_of(fre_ctx *c) { return fre::ctx_launch(c); }

// phi and mu of the current state into phi[1 - pp] and mu.
void current_phi_mu(fre_ctx *c, const fre::Launch &L) {
    c->ks->phi(L, !c->local);
    if (c->n_ghost) fre::ghost_fields(c, L, false);
    c->ks->mu(L);
    if (c->n_ghost) fre::ghost_fields(c, L, true);
}

fre_status check_launch(const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FRE_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return FRE_OK;
}

// After a synchronisation: report a kernel whose bounded wait timed out.
fre_status check_device_error(fre_ctx *c) {
    int e = 0;
    if (cudaMemcpy(&e, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FRE_ERR_CUDA, "reading the device error word: %s", cudaGetErrorString(cudaGetLastError()));
    if (e) {
        cudaMemset(c->err_dev, 0, sizeof(int));
        return fail(FRE_ERR_CUDA, "a pipelined kernel gave up waiting for its bulk copies (code %d)", e);
    }
    return FRE_OK;
}

fre_status ensure_staging(fre_ctx *c) {
    if (c->staging) return FRE_OK;
    void *p = nullptr;
    fre_status s = dev_alloc(c, &p, sizeof(double) * 6 * (size_t)c->G.n);
    if (s != FRE_OK) return s;
    c->staging = static_cast<double *>(p);
    return FRE_OK;
}

fre_status ensure_ccl(fre_ctx *c) {
    if (c->ccl.labels) return FRE_OK;
    const size_t n = (size_t)c->G.n;
    void *p = nullptr;
    fre_status s = dev_alloc(c, &p, 2 * sizeof(int) * n + 16 * (size_t)kCclCap + 256);
    if (s != FRE_OK) return s;
    char *b = static_cast<char *>(p);
    c->ccl.pairs = reinterpret_cast<long long *>(b);
    c->ccl.count = reinterpret_cast<int *>(b + 16 * (size_t)kCclCap);
    c->ccl.labels = reinterpret_cast<int *>(b + 16 * (size_t)kCclCap + 256);
    c->ccl.sizes = c->ccl.labels + n;
    c->ccl.cap = kCclCap;
    return FRE_OK;
}

fre_status enter(fre_ctx *c) {
    if (!c) return fail(FRE_ERR_ARG, "context is NULL");
    FRE_CUDA(cudaSetDevice(c->device_id));
    return FRE_OK;
}

// phi field set -> ghosts -> mu -> ghosts -> equilibria into buffer 0
fre_status finish_init(fre_ctx *c, int from_staging) {
    c->cur = 0;
    c->pp = 1;
    fre::Launch L = launch_of(c);  // phi = phi[0], src = buf[0]
    if (c->n_ghost) fre::ghost_fields(c, L, false);
    c->ks->mu(L);
    if (c->n_ghost) fre::ghost_fields(c, L, true);
    c->ks->init_eq(L, from_staging);
    fre_status s = check_launch("init");
    if (s != FRE_OK) return s;
    c->local = true;
    c->initialised = true;
    c->step = 0;
    return FRE_OK;
}

}  // namespace

namespace fre {
void set_last_error(const char *msg) { g_err = msg ? msg : ""; }
}  // namespace fre

extern "C" {

size_t fre_device_bytes(const fre_params *p) {
    Sizes s;
    if (!sizes_of(p, s, nullptr)) return 0;
    return total_bytes(s);
}

fre_status fre_create(const fre_params *p, void *cuda_stream, fre_ctx **out) {
    if (!out) return fail(FRE_ERR_ARG, "out is NULL");
    *out = nullptr;
    Sizes s;
    std::string why;
    if (!sizes_of(p, s, &why)) return fail(FRE_ERR_ARG, "fre_create: %s", why.c_str());
    fre_ctx *c = new fre_ctx();
    c->p = *p;
    c->q = s.q;
    auto bail = [&](fre_status st) {
        fre_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device_id) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(FRE_ERR_CUDA, "fre_create: no CUDA device");
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return fail(FRE_ERR_CUDA, "fre_create: cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    c->ks = p->lattice == FRE_D2Q9 ? fre::kernels_d2q9(p->precision) : fre::kernels_d3q19(p->precision);
    c->G.nx = p->nx;
    c->G.ny = p->ny;
    c->G.nz = p->nz;
    c->G.device = p->device;
    c->G.n = s.n;
    c->G.np = s.np;
    c->G.uwall = p->u_wall;
    c->P = {p->tau_f, p->tau_g, p->A, p->kappa, p->gamma_mob, p->rho0, p->model, p->kappa1, p->kappa2, p->alpha};

    const bool dev16 = p->precision == FRE_FP16DEV || p->precision == FRE_BF16DEV;
    const size_t plane = (size_t)s.np * s.sz_store;
    for (int b = 0; b < 2; ++b) {
        void *ptr;
        fre_status st = dev_alloc(c, &ptr, s.buf_bytes);
        if (st != FRE_OK) return bail(st);
        char *base = static_cast<char *>(ptr);
        c->buf[b].f = base;
        c->buf[b].g = base + (size_t)s.q * plane;
        c->buf[b].g0 = dev16 ? reinterpret_cast<float *>(base + (size_t)(2 * s.q - 1) * plane) : nullptr;
    }
    for (int k = 0; k < 2; ++k) {
        fre_status st = dev_alloc(c, &c->phi[k], s.field_bytes);
        if (st != FRE_OK) return bail(st);
    }
    {
        fre_status st = dev_alloc(c, &c->mu, s.field_bytes);
        if (st != FRE_OK) return bail(st);
        if (p->model == 1) {
            st = dev_alloc(c, &c->rhof, s.field_bytes);
            if (st != FRE_OK) return bail(st);
            st = dev_alloc(c, &c->murho, s.field_bytes);
            if (st != FRE_OK) return bail(st);
        }
        void *r;
        st = dev_alloc(c, &r, sizeof(double) * fre::kRedDoublesHost);
        if (st != FRE_OK) return bail(st);
        c->red = static_cast<double *>(r);
        void *o;
        st = dev_alloc(c, &o, sizeof(fre_obs));
        if (st != FRE_OK) return bail(st);
        c->obs_dev = static_cast<fre_obs *>(o);
        void *e;
        st = dev_alloc(c, &e, sizeof(int) * 4);
        if (st != FRE_OK) return bail(st);
        c->err_dev = static_cast<int *>(e);
    }
    long long rb = (s.n + 255) / 256;
    c->red_blocks = (int)(rb < 608 ? (rb < 1 ? 1 : rb) : 608);
    if (cudaMallocHost(&c->obs_host, sizeof(fre_obs)) != cudaSuccess) {
        cudaGetLastError();
        c->obs_host = nullptr;
        return bail(fail(FRE_ERR_OOM, "cudaMallocHost failed"));
    }
    if (p->device == FRE_FOUR_ROLLER) {
        std::vector<unsigned char> solid;
        std::vector<int> ghost;
        std::vector<int4> links, linkq;
        build_rollers(c, solid, ghost, links, linkq);
        void *d;
        fre_status st = dev_alloc(c, &d, s.solid_bytes);
        if (st != FRE_OK) return bail(st);
        c->solid = static_cast<unsigned char *>(d);
        if (cudaMemcpyAsync(c->solid, solid.data(), solid.size(), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            return bail(fail(FRE_ERR_CUDA, "upload of the roller mask failed"));
        c->n_ghost = (int)ghost.size();
        if (c->n_ghost) {
            st = dev_alloc(c, &d, sizeof(int) * ghost.size());
            if (st != FRE_OK) return bail(st);
            c->ghost = static_cast<int *>(d);
            if (cudaMemcpyAsync(c->ghost, ghost.data(), sizeof(int) * ghost.size(), cudaMemcpyHostToDevice,
                                c->stream) != cudaSuccess)
                return bail(fail(FRE_ERR_CUDA, "upload of the ghost list failed"));
        }
        c->n_rlinks = (int)links.size();
        if (c->n_rlinks) {
            st = dev_alloc(c, &d, sizeof(int4) * links.size());
            if (st != FRE_OK) return bail(st);
            c->rlinks = static_cast<int4 *>(d);
            if (cudaMemcpyAsync(c->rlinks, links.data(), sizeof(int4) * links.size(), cudaMemcpyHostToDevice,
                                c->stream) != cudaSuccess)
                return bail(fail(FRE_ERR_CUDA, "upload of the roller links failed"));
        }
        if (!linkq.empty()) {
            st = dev_alloc(c, &d, sizeof(int4) * linkq.size());
            if (st != FRE_OK) return bail(st);
            c->rlinkq = static_cast<int4 *>(d);
            if (cudaMemcpyAsync(c->rlinkq, linkq.data(), sizeof(int4) * linkq.size(), cudaMemcpyHostToDevice,
                                c->stream) != cudaSuccess)
                return bail(fail(FRE_ERR_CUDA, "upload of the roller link fractions failed"));
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess)
            return bail(fail(FRE_ERR_CUDA, "geometry upload: %s", cudaGetErrorString(cudaGetLastError())));
    }
    c->G.solid = c->solid;
    c->G.rlinks = c->rlinks;
    c->G.n_rlinks = c->n_rlinks;
    c->G.rlinkq = c->rlinkq;
    // the full functional (model 1) runs on the per-node kernels; the
    // interpolated roller walls take the row kernels with the interpolating
    // reflection pass (FP32 and 16-bit storage)
    const bool per_node = (p->flags & FRE_FLAG_GENERIC_KERNELS) || p->model != 0;
    if (!per_node && c->ks->row_width) {
        const unsigned sh = (p->flags >> FRE_FLAG_CHUNK_SHIFT) & 0xffu;
        c->row_w = c->ks->row_width(c->G, sh ? (1 << sh) : 0);
        c->rows = c->row_w > 0;
    }
    // the four-roller device has no chunked row kernels, only full rows
    c->fullrow = !per_node && (c->rows || p->device == FRE_FOUR_ROLLER) &&
                 !(p->flags & FRE_FLAG_CHUNKED_UPDATE) && c->ks->fullrow_usable && c->ks->fullrow_usable(c->G);
    cudaGetLastError();
    *out = c;
    return FRE_OK;
}

fre_status fre_init_droplet(fre_ctx *c, double cx, double cy, double cz, double R) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (c->p.model == 0 && (!(c->p.A > 0.0) || !(c->p.kappa > 0.0)))
        return fail(FRE_ERR_ARG, "fre_init_droplet needs A > 0, kappa > 0");
    if (c->p.model == 1 && !(c->p.alpha > 0.0)) return fail(FRE_ERR_ARG, "fre_init_droplet needs alpha > 0");
    if (!(R > 0.0) || !std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(cz))
        return fail(FRE_ERR_ARG, "fre_init_droplet: R must be > 0 and the centre finite");
    c->cur = 0;
    c->pp = 1;
    fre::Launch L = launch_of(c);
    L.phi = c->phi[0];
    c->ks->set_phi(L, 1, cx, cy, cz, R);
    return finish_init(c, 0);
}

fre_status fre_init_fields(fre_ctx *c, const double *rho, const double *ux, const double *uy, const double *uz,
                           const double *phi) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!rho || !ux || !uy || !phi) return fail(FRE_ERR_ARG, "fre_init_fields: rho, ux, uy, phi are required");
    if (c->p.lattice == FRE_D3Q19 && !uz) return fail(FRE_ERR_ARG, "fre_init_fields: D3Q19 needs uz");
    s = ensure_staging(c);
    if (s != FRE_OK) return s;
    const size_t N = (size_t)c->G.n, bytes = N * sizeof(double);
    const double *src[5] = {rho, ux, uy, uz, phi};
    for (int k = 0; k < 5; ++k) {
        if (src[k]) {
            FRE_CUDA(cudaMemcpyAsync(c->staging + k * N, src[k], bytes, cudaMemcpyHostToDevice, c->stream));
        } else {
            FRE_CUDA(cudaMemsetAsync(c->staging + k * N, 0, bytes, c->stream));
        }
    }
    c->cur = 0;
    c->pp = 1;
    fre::Launch L = launch_of(c);
    L.phi = c->phi[0];
    c->ks->set_phi(L, 0, 0, 0, 0, 0);
    s = finish_init(c, 1);
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    return FRE_OK;
}

fre_status fre_init_consistent(fre_ctx *c, int iterations) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (iterations < 0) return fail(FRE_ERR_ARG, "fre_init_consistent: iterations < 0");
    if (!c->initialised || !c->local || c->step != 0)
        return fail(FRE_ERR_STATE, "fre_init_consistent: call it right after an initialisation or a load");
    s = ensure_staging(c);
    if (s != FRE_OK) return s;
    fre::Launch L = launch_of(c);
    current_phi_mu(c, L);  // phi0, mu0 (and roller ghosts) of the in-place state
    c->ks->mei_prep(L);
    bool pull = false;
    for (int it = 0; it < iterations; ++it) {
        L = launch_of(c);
        c->ks->mei_iter(L, pull);
        c->cur ^= 1;
        pull = true;
    }
    L = launch_of(c);
    c->ks->mei_final(L, pull);
    c->cur ^= 1;
    c->local = true;
    c->step = 0;
    s = check_launch("fre_init_consistent");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

fre_status fre_load_populations(fre_ctx *c, const double *f, const double *g) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!f || !g) return fail(FRE_ERR_ARG, "fre_load_populations: f and g are required");
    s = ensure_staging(c);
    if (s != FRE_OK) return s;
    c->cur = 0;
    c->pp = 1;
    fre::Launch L = launch_of(c);
    const size_t N = (size_t)c->G.n;
    for (int lat = 0; lat < 2; ++lat) {
        const double *h = lat ? g : f;
        for (int i = 0; i < c->q; ++i) {
            FRE_CUDA(cudaMemcpyAsync(c->staging, h + i * N, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            c->ks->load_plane(L, lat, i);
        }
    }
    s = check_launch("fre_load_populations");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    c->local = true;
    c->initialised = true;
    c->step = 0;
    return FRE_OK;
}

fre_status fre_store_populations(fre_ctx *c, double *f, double *g) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_store_populations: not initialised");
    s = ensure_staging(c);
    if (s != FRE_OK) return s;
    fre::Launch L = launch_of(c);
    const size_t N = (size_t)c->G.n;
    for (int lat = 0; lat < 2; ++lat) {
        double *h = lat ? g : f;
        if (!h) continue;
        for (int i = 0; i < c->q; ++i) {
            c->ks->pull_plane(L, !c->local, lat, i);
            FRE_CUDA(cudaMemcpyAsync(h + i * N, c->staging, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        }
    }
    s = check_launch("fre_store_populations");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

fre_status fre_step(fre_ctx *c, int nsteps) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (nsteps < 0) return fail(FRE_ERR_ARG, "fre_step: nsteps < 0");
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_step: not initialised");
    for (int t = 0; t < nsteps; ++t) fre::ctx_launch_step(c);
    return check_launch("fre_step");
}

fre_status fre_step_timed(fre_ctx *c, int nsteps, double *ms, long long *launches) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (nsteps < 0 || !ms) return fail(FRE_ERR_ARG, "fre_step_timed: nsteps < 0 or ms is NULL");
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_step_timed: not initialised");
    std::vector<cudaEvent_t> ev((size_t)3 * nsteps + 1);
    for (auto &e : ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return fail(FRE_ERR_CUDA, "fre_step_timed: cudaEventCreate failed");
        }
    }
    long long nl = 0;
    cudaEventRecord(ev[0], c->stream);
    for (int t = 0; t < nsteps; ++t) {
        fre::Launch L = launch_of(c);
        const bool pull = !c->local;
        const bool full = c->fullrow && (pull || c->G.device != FRE_FOUR_ROLLER);
        if (full) c->ks->phi_fullrow(L, pull);
        else if (c->rows) c->ks->phi_rows(L, pull);
        else c->ks->phi(L, pull);
        ++nl;
        cudaEventRecord(ev[3 * t + 1], c->stream);
        if (c->n_ghost) { fre::ghost_fields(c, L, false); nl += 1 + c->P.model; }
        if (full) c->ks->mu_fullrow(L);
        else if (c->rows) c->ks->mu_rows(L);
        else c->ks->mu(L);
        ++nl;
        if (c->n_ghost) { fre::ghost_fields(c, L, true); nl += 1 + c->P.model; }
        cudaEventRecord(ev[3 * t + 2], c->stream);
        if (full) c->ks->update_fullrow(L, pull);
        else if (c->rows) c->ks->update_rows(L, pull);
        else c->ks->update(L, pull);
        ++nl;
        if ((full || (c->fullrow && c->G.interp)) && c->G.device == FRE_FOUR_ROLLER) {
            c->ks->reflect(L);
            ++nl;
        }
        cudaEventRecord(ev[3 * t + 3], c->stream);
        c->cur ^= 1;
        c->pp ^= 1;
        c->local = false;
        c->step++;
    }
    s = check_launch("fre_step_timed");
    cudaError_t e = cudaEventSynchronize(ev.back());
    for (int k = 0; k < 4; ++k) ms[k] = 0.0;
    if (s == FRE_OK && e == cudaSuccess) {
        for (int t = 0; t < nsteps; ++t)
            for (int k = 0; k < 3; ++k) {
                float x = 0.f;
                cudaEventElapsedTime(&x, ev[3 * t + k], ev[3 * t + k + 1]);
                ms[k] += x;
            }
        float tot = 0.f;
        cudaEventElapsedTime(&tot, ev[0], ev.back());
        ms[3] = tot;
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (launches) *launches = nl;
    if (s != FRE_OK) return s;
    if (e != cudaSuccess) return fail(FRE_ERR_CUDA, "fre_step_timed: %s", cudaGetErrorString(e));
    return check_device_error(c);
}

fre_status fre_copy_fields(fre_ctx *c, double *rho, double *ux, double *uy, double *uz, double *phi, double *mu) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_copy_fields: not initialised");
    s = ensure_staging(c);
    if (s != FRE_OK) return s;
    fre::Launch L = launch_of(c);
    current_phi_mu(c, L);
    c->ks->macro(L, !c->local);
    double *dst[6] = {rho, ux, uy, uz, phi, mu};
    const size_t N = (size_t)c->G.n;
    for (int k = 0; k < 6; ++k)
        if (dst[k])
            FRE_CUDA(cudaMemcpyAsync(dst[k], c->staging + k * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                                     c->stream));
    s = check_launch("fre_copy_fields");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

fre_status fre_observables(fre_ctx *c, fre_obs *out) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!out) return fail(FRE_ERR_ARG, "fre_observables: out is NULL");
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_observables: not initialised");
    fre::Launch L = launch_of(c);
    current_phi_mu(c, L);
    c->ks->obs(L, !c->local);
    FRE_CUDA(cudaMemcpyAsync(c->obs_host, c->obs_dev, sizeof(fre_obs), cudaMemcpyDeviceToHost, c->stream));
    s = check_launch("fre_observables");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    s = check_device_error(c);
    if (s != FRE_OK) return s;
    *out = *c->obs_host;
    out->step = c->step;
    if (out->status != 0)
        return fail(FRE_ERR_UNSTABLE, "fre_observables: %s", out->status == 1 ? "non-finite values" : "|u| > 0.3");
    return FRE_OK;
}

fre_status fre_components(fre_ctx *c, long long min_size, int *count, long long *sizes, int max_sizes, int *labels) {
    fre_status s = enter(c);
    if (s != FRE_OK) return s;
    if (!count || max_sizes < 0 || (max_sizes > 0 && !sizes))
        return fail(FRE_ERR_ARG, "fre_components: count is NULL, or sizes is NULL with max_sizes > 0");
    if (!c->initialised) return fail(FRE_ERR_STATE, "fre_components: not initialised");
    s = ensure_ccl(c);
    if (s != FRE_OK) return s;
    fre::Launch L = launch_of(c);
    current_phi_mu(c, L);
    fre::ccl_label(L, c->p.lattice, c->p.precision, min_size < 1 ? 1 : min_size, c->ccl);
    int nroots = 0;
    FRE_CUDA(cudaMemcpyAsync(&nroots, c->ccl.count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    s = check_launch("fre_components");
    if (s != FRE_OK) return s;
    FRE_CUDA(cudaStreamSynchronize(c->stream));
    *count = nroots;
    if (max_sizes > 0) {
        const int k = nroots < c->ccl.cap ? nroots : c->ccl.cap;
        std::vector<long long> pairs(2 * (size_t)k);
        if (k) FRE_CUDA(cudaMemcpy(pairs.data(), c->ccl.pairs, sizeof(long long) * 2 * (size_t)k,
                                   cudaMemcpyDeviceToHost));
        std::vector<long long> sz(k);
        for (int j = 0; j < k; ++j) sz[j] = pairs[2 * (size_t)j];
        std::sort(sz.begin(), sz.end(), [](long long a, long long b) { return a > b; });
        for (int j = 0; j < max_sizes; ++j) sizes[j] = j < k ? sz[j] : 0;
    }
    if (labels)
        FRE_CUDA(cudaMemcpy(labels, c->ccl.labels, sizeof(int) * (size_t)c->G.n, cudaMemcpyDeviceToHost));
    return check_device_error(c);
}

long long fre_step_count(const fre_ctx *c) { return c ? c->step : -1; }

int fre_uses_row_kernels(const fre_ctx *c) { return c && (c->rows || c->fullrow) ? 1 : 0; }

int fre_kernel_path(const fre_ctx *c) { return !c ? -1 : (c->fullrow ? 2 : (c->rows ? 1 : 0)); }

void fre_destroy(fre_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device_id);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void *p : c->allocs) cudaFree(p);
    if (c->obs_host) cudaFreeHost(c->obs_host);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

const char *fre_last_error(void) { return g_err.c_str(); }

}  // extern "C"
