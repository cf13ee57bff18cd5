// Internal types shared by the host runtime (fre_api.cu) and the kernel
// translation units (fre_d2q9.cu, fre_d3q19.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/fre.h"

namespace fre {

// Geometry of one lattice: sizes, device kind and the analytic walls.
struct Geo {
    int nx, ny, nz, device;
    long long n;              // nodes
    long long np;             // plane stride of the population arrays (elements)
    const unsigned char *solid;  // roller id per node (0 = fluid); four-roller only
    // four-roller: the wall links of one z plane (every plane has the same,
    // the rollers being extruded along z), for the reflection pass of the
    // row kernels (k_reflect): {fluid node y nx + x, its link's roller
    // source (wrapped) y' nx + x', i | opp(i) << 8 | (c_iz + 1) << 16,
    // float bits of 2 w_i (c_i . u_w) / cs^2}
    const int4 *rlinks;
    int n_rlinks;
    // interpolated roller walls on the row kernels: per entry of rlinks,
    // {float bits of the fraction q of the link from the fluid node toward
    // its roller source that lies outside the roller circle, the fluid
    // node's neighbour x + c_i in the plane (y nx + x, wrapped), 1 if that
    // neighbour is a roller node, 0}; nullptr otherwise
    const int4 *rlinkq;
    double rcx[5], rcy[5], om[5];  // roller centres and angular velocities (1..4)
    double rr;                // roller radius
    int interp;               // four-roller: interpolated bounce-back at the roller surfaces
    double uwall;             // shear wall speed
};

// Physical parameters of the scheme (Sec. 2.2).
struct Phys {
    double tau_f, tau_g, A, kappa, Gamma, rho0;
    int model;  // 0 reduced functional; 1 the full functional of kappa1, kappa2, alpha
    double kappa1, kappa2, alpha;
};

// FP32 copies of the per-launch constants of the FP32-compute kernels,
// rounded once on the host: the GPU's FP64 pipe is narrow, so the kernels
// do no double arithmetic per work unit or node.  u0, du: the reference
// profile U(y) = u0 + y du of the 16-bit f stores (fref in fre_kernels.cuh):
// the plane Couette profile of the shear device unless
// FRE_FLAG_REST_REFERENCE, else 0 (the rest equilibrium).
struct PhysF {
    float omega_f, omega_g, kf, gamma3, A, kappa, rho0, uwall, u0, du;
    float rcx[5], rcy[5], rom[5];  // four-roller: roller centres and angular velocities
};

// One population buffer (A or B).  FP64/FP32: f, g are [q][np] arrays of
// the storage type.  16-bit formats: f is [q][np] of deviations
// f_i - fr_i(y) from the reference of the node's row (fref in
// fre_kernels.cuh; the Couette equilibrium of the shear device, else w_i rho0); g holds
// g_1..g_{q-1} as [q-1][np]; g0 is FP32 [np].
struct Buf {
    void *f;
    void *g;
    float *g0;
};

// Everything a kernel launch needs.  phi/mu are arrays of the compute type.
struct Launch {
    Geo G;
    Phys P;
    PhysF F;
    Buf src, dst;
    const void *phi_prev;  // phi at the previous step (moving-wall term of g)
    void *phi;             // phi at the current step
    void *mu;              // mu at the current step (model 1: mu_phi)
    void *rhof;            // model 1: rho at the current step
    void *murho;           // model 1: mu_rho at the current step
    const int *ghost;      // roller solid nodes with fluid neighbours
    int n_ghost;
    double *red;           // reduction scratch
    int red_blocks;
    fre_obs *obs;          // device observables
    int W;                 // chunk width of the row kernels
    int pull;              // batched kernels: stream from the post-collision buffer
    int *err;              // device error word (pipeline wait timed out)
    unsigned long long wait_ns;  // limit of every pipeline wait
    int stall;             // FRE_FLAG_TEST_PIPELINE_STALL: producers issue no copies
    int reflect;           // four-roller on the row kernels: per-node updates also
                           // reflect their wall links into the roller nodes' slots
                           // (the row update leaves that to k_reflect)
    double *staging;       // FP64 staging of host I/O (n doubles per field)
    cudaStream_t stream;
};

// Per lattice and storage format: the kernels of one time step and of the
// I/O paths.  `pull` selects streaming from the post-collision buffer (true)
// or reading pre-collision populations in place (false, right after an
// initialisation or a load).
struct KernelSet {
    void (*phi)(const Launch &, bool pull);           // phi = sum g (pulled)
    void (*ghost)(const Launch &, void *field);       // roller solid stencil values
    void (*mu)(const Launch &);                        // mu from phi
    void (*update)(const Launch &, bool pull);        // fused pull + collide
    void (*obs)(const Launch &, bool pull);           // observables -> L.obs
    void (*macro)(const Launch &, bool pull);         // rho,u,phi,mu -> staging
    void (*pull_plane)(const Launch &, bool pull, int lattice_g, int i);  // -> staging
    void (*load_plane)(const Launch &, int lattice_g, int i);  // staging -> src
    void (*set_phi)(const Launch &, int analytic, double cx, double cy, double cz, double R);
    void (*init_eq)(const Launch &, int from_staging);  // f = f_eq, g = g_eq into src
    // consistent initialisation: u0 and F0 of the in-place state into
    // staging; one collide(u0, F0 held)-and-stream pass of f src -> dst; the
    // pulled f and g = g_eq(phi, mu, u0) into dst as the pre-collision state
    void (*mei_prep)(const Launch &);
    void (*mei_iter)(const Launch &, bool pull);
    void (*mei_final)(const Launch &, bool pull);
    // row kernels of the hot path (nullptr where the format has none)
    int (*row_width)(const Geo &, int pref);  // chunk width of the row kernels, 0 = n/a
    void (*phi_rows)(const Launch &, bool pull);
    void (*mu_rows)(const Launch &);
    void (*update_rows)(const Launch &, bool pull);
    // full-row variant of the update (one bulk copy per population row)
    bool (*fullrow_usable)(const Geo &);
    void (*update_fullrow)(const Launch &, bool pull);
    void (*phi_fullrow)(const Launch &, bool pull);
    void (*mu_fullrow)(const Launch &);
    // four-roller device on the row kernels: after the update, the wall
    // links of the step reflected into the roller nodes' slots of dst
    void (*reflect)(const Launch &);
};

// Many contexts of one lattice and storage format advanced by one launch
// per kernel: per-slot launch descriptors and block tables on the device.
struct BatchLaunch {
    const Launch *cases;     // [nslots]
    const int *block_start;  // [nslots + 1], exclusive prefix of lattice blocks
    const int *ghost_start;  // [nslots + 1], exclusive prefix of ghost blocks
    int nslots;
    int total_blocks;
    int total_ghost_blocks;
    cudaStream_t stream;
};

// Batched per-node kernels, templated on the block width BX (BY = 256/BX).
struct BatchKernels {
    void (*phi)(const BatchLaunch &, int bx);
    void (*mu)(const BatchLaunch &, int bx);
    void (*ghost)(const BatchLaunch &, int field);  // field 0: phi, 1: mu
    void (*update)(const BatchLaunch &, int bx);
};

const BatchKernels *batch_kernels_d2q9(int precision);
const BatchKernels *batch_kernels_d3q19(int precision);

// Device buffers of the component labelling (fre_components): labels and
// sizes [n], a count and up to `cap` (size, root) pairs.
struct CclBuffers {
    int *labels;
    int *sizes;
    int *count;
    long long *pairs;
    int cap;
};
// Label the connected components of the phase phi > 0 of L.phi (fre_ccl.cu)
// and list the roots of those with at least min_size nodes; queued on
// L.stream.
void ccl_label(const Launch &L, int lattice, int precision, long long min_size, const CclBuffers &B);

const KernelSet *kernels_d2q9(int precision);
const KernelSet *kernels_d3q19(int precision);

// Record the message returned by fre_last_error() on this thread.
void set_last_error(const char *msg);

}  // namespace fre
