/*
 * fre.h -- C ABI of the GB300 (sm_103a) two-lattice free energy lattice
 * Boltzmann update (Simonis et al., arXiv:2212.01617).
 *
 * One context holds one simulation: the momentum populations f (Eq. LBE) and
 * the order-parameter populations g (Eq. LBEg) on a D2Q9 or D3Q19 lattice,
 * resident in device memory, plus the auxiliary phi and mu fields.  Each
 * time step (fre_step) runs, on the device and in the paper's order
 * (Algorithm 1, Sec. 2.3):
 *   rho = sum f_i, phi = sum g_i            (Eq. densMoment, Eq. ordeMoment)
 *   mu  = A(phi^3 - phi) - kappa lap(phi)   (Eq. mu_phi, kappa_1 = kappa_2,
 *                                            rho = 1; isotropic stencil)
 *   F   = -phi grad(mu)                     (Eq. F without the rho term;
 *                                            evaluated as mu grad(phi) -
 *                                            grad(phi mu))
 *   u   = (sum c_i f_i + F/2) / rho         (Eq. veloMoment)
 *   BGK + Guo for f, BGK for g              (Eq. bgk, Eq. feq, Eq. Fi,
 *                                            Eq. geq, Eq. LBEg)
 *   streaming with half-way bounce-back and the moving-wall term at solid
 *   sources (the usual LBM wall treatment the paper defers to, Sec. 2.3).
 *
 * Conventions shared by every entry point:
 *   - node index n = (z*ny + y)*nx + x, x fastest; D2Q9 has nz = 1;
 *   - host population arrays are FP64 [q][n] in this direction order
 *       D2Q9 : 0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1); 5 (1,1);
 *              6 (-1,1); 7 (-1,-1); 8 (1,-1)
 *       D3Q19: 0 rest; 1 (1,0,0); 2 (-1,0,0); 3 (0,1,0); 4 (0,-1,0);
 *              5 (0,0,1); 6 (0,0,-1); 7 (1,1,0); 8 (-1,-1,0); 9 (1,0,1);
 *              10 (-1,0,-1); 11 (0,1,1); 12 (0,-1,-1); 13 (1,-1,0);
 *              14 (-1,1,0); 15 (1,0,-1); 16 (-1,0,1); 17 (0,1,-1);
 *              18 (0,-1,1)
 *     and hold the PRE-collision populations f(x,t), g(x,t);
 *   - host pointers are owned by the caller and only read/written during the
 *     call; all device memory is owned by the context;
 *   - every call returns a fre_status and never aborts; fre_last_error()
 *     gives a human-readable message for the last failure of this thread;
 *   - calls on one context must not overlap (one host thread at a time);
 *     the work is issued on the context's CUDA stream.
 */
#ifndef FRE_H
#define FRE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FRE_OK = 0,
    FRE_ERR_ARG = 1,       /* invalid argument (checked before any work) */
    FRE_ERR_OOM = 2,       /* device allocation failed */
    FRE_ERR_CUDA = 3,      /* a CUDA call failed; the context is unusable */
    FRE_ERR_UNSTABLE = 4,  /* non-finite values or |u| > 0.3 were found */
    FRE_ERR_BUDGET = 5,    /* admission refused: device-memory budget */
    FRE_ERR_STATE = 6      /* call not valid in the current state */
} fre_status;

typedef enum { FRE_D2Q9 = 0, FRE_D3Q19 = 1 } fre_lattice;

/* Storage of the populations on the device.  FP64 and FP32 store f_i and
 * g_i as is and compute in the same precision.  FP16DEV and BF16DEV store
 * f_i - fr_i, the deviation from a reference equilibrium (the Couette
 * equilibrium of the shear device, w_i rho0 elsewhere; see
 * FRE_FLAG_REST_REFERENCE), and g_i (i != 0) in 16 bits (round to nearest
 * even), keep g_0 in FP32 and compute in FP32. */
typedef enum { FRE_FP64 = 0, FRE_FP32 = 1, FRE_FP16DEV = 2, FRE_BF16DEV = 3 } fre_precision;

/* FRE_SHEAR: Taylor's parallel-band device (Sec. 3.1): walls at y = -1/2
 *   (moving at -u_wall in x) and y = ny - 1/2 (moving at +u_wall), periodic
 *   in x and z.
 * FRE_FOUR_ROLLER: Taylor's four-roller device (Sec. 3.2): four staircase
 *   cylinders (axis z) of radius nx/8 centred at ((nx-1)/2 +- nx/4,
 *   (ny-1)/2 +- ny/4) with surface speed u_wall, top-right and bottom-left
 *   counter-clockwise, the others clockwise, so the centre sees extension
 *   along x; periodic outer box.
 * FRE_PERIODIC: fully periodic box (no walls). */
typedef enum { FRE_SHEAR = 0, FRE_FOUR_ROLLER = 1, FRE_PERIODIC = 2 } fre_device;

typedef struct {
    int lattice;       /* fre_lattice */
    int precision;     /* fre_precision */
    int device;        /* fre_device */
    int nx, ny, nz;    /* lattice nodes; nz = 1 for D2Q9; each >= 1 */
    double tau_f;      /* relaxation time of f, > 0.5 (Eq. bgk) */
    double tau_g;      /* relaxation time of g, > 0.5 (Eq. LBEg) */
    double A;          /* bulk free-energy coefficient, >= 0 */
    double kappa;      /* gradient free-energy coefficient, >= 0 */
    double gamma_mob;  /* mobility parameter Gamma (Eq. geq), M = Gamma (tau_g - 1/2) */
    double u_wall;     /* wall (shear) or roller surface (four-roller) speed */
    double rho0;       /* reference density; also the wall density of the
                          moving bounce-back term */
    unsigned flags;    /* FRE_FLAG_* bits, 0 by default */
    /* Free-energy model.  0 (default): the reduced functional of A and kappa
     * above, mu = A(phi^3 - phi) - kappa lap(phi), force -phi grad(mu).
     * 1: the paper's full functional (Eq. functional) of kappa1, kappa2 and
     * alpha, with mu_rho and mu_phi (Eq. mu_rho, Eq. mu_phi) and the force
     * -rho grad(mu_rho) - phi grad(mu_phi) (Eq. F); A and kappa are then
     * unused.  Its planar interface is tanh(x / (2 alpha)) (xi = sqrt(2)
     * alpha) and its interface tension alpha (kappa1 + kappa2) / 6; with
     * kappa1 = kappa2 = kappa_p it reduces to model 0 with A = kappa_p / 4,
     * kappa = alpha^2 kappa_p / 2 at rho = 1.  Model 1 runs on the per-node
     * kernels and is not taken by batches and servers. */
    int model;
    double kappa1, kappa2, alpha;
} fre_params;

/* Force the per-node kernels even where the row kernels apply (the row
 * kernels stage whole x-rows in shared memory; both compute the same
 * update).  For validation. */
#define FRE_FLAG_GENERIC_KERNELS 1u
/* Run the update on x-chunk work units instead of whole x-rows (both stage
 * their rows in shared memory with bulk copies; for validation/tuning). */
#define FRE_FLAG_CHUNKED_UPDATE 2u
/* Reference state of the 16-bit f stores on the shear device.  By default
 * f_i is stored as the deviation from the equilibrium (Eq. feq) of rho0 and
 * the plane Couette velocity between the walls, (U(y), 0, 0) with U(y) =
 * u_wall (2 (y + 1/2) / ny - 1): the base flow the moving walls drive, the
 * state of the device before a droplet deforms it.  The 16-bit values then
 * carry the departure from that base flow only.  FRE_FLAG_REST_REFERENCE
 * stores f_i - w_i rho0 instead, the deviation from the equilibrium at rest;
 * every moving f_i then also carries the base flow 3 w_i rho0 c_ix U(y), on
 * which FP16 spends its mantissa (on the 64^3 shear twin of the benchmark
 * lattice the FP16 error in D is 3.2e-3 with the rest reference and 4.1e-5
 * with the Couette one, at the same speed).  FRE_FLAG_COUETTE_REFERENCE
 * names the default; setting both is an argument error.  FP64, FP32 and
 * the devices without moving walls ignore both (their reference is
 * w_i rho0). */
#define FRE_FLAG_COUETTE_REFERENCE 4u
#define FRE_FLAG_REST_REFERENCE 8u
/* Test of the failure path of the row kernels, not for production: their
 * producer warps issue no copies and every pipeline wait gives up after
 * 5 ms instead of 2 s.  Each step's kernels then end early with the
 * context's error word set, and the next synchronising call (fre_observables,
 * fre_copy_fields, fre_store_populations, fre_step_timed) returns
 * FRE_ERR_CUDA; the GPU and other contexts are unaffected.  The populations
 * of such a context are left undefined: initialise it again before use. */
#define FRE_FLAG_TEST_PIPELINE_STALL 16u
/* Four-roller device only (an argument error elsewhere): bounce-back at the
 * roller surfaces interpolated along each wall link instead of half-way
 * bounce-back on the staircase of roller nodes.  The circle cuts the link
 * from a fluid node x toward its roller source x - c_i at x - q c_i,
 * 0 < q <= 1; the linear rule of Bouzidi, Firdaouss and Lallemand (Phys.
 * Fluids 13, 2001) then gives the pulled population
 *   q < 1/2:  2q f*_ibar(x) + (1 - 2q) f*_ibar(x + c_i) + m_i
 *             (half-way bounce-back f*_ibar(x) + m_i where x + c_i is a
 *             roller node too),
 *   q >= 1/2: [f*_ibar(x) + (2q - 1) f*_i(x) + m_i] / (2q),
 * with the moving-wall term m_i = 2 w_i rho0 (c_i . u_w) / cs^2 of the
 * roller's rotation (g alike, with phi(x, t) in place of rho0).  The wall
 * then sits on the circle to second order instead of on the staircase.
 * FP64 runs it on the per-node kernels; FP32 and 16-bit storage on the row
 * kernels, where a pass after each update writes every link's value into
 * its roller source (link fractions computed once, in double, at create).
 * Batches and servers do not take it. */
#define FRE_FLAG_INTERPOLATED_WALLS 32u
/* Bits 8..15: log2 of the x-chunk width of the row kernels (0 = automatic:
 * 128 when nx allows it, else the whole row).  A tuning knob; every valid
 * width computes the same update. */
#define FRE_FLAG_CHUNK_SHIFT 8

/* Observables of the state at the current step, from the pre-collision
 * populations; sums in FP64 over fluid nodes. */
typedef struct {
    double mass;         /* sum rho */
    double phi_sum;      /* sum phi */
    double volume;       /* sum (1 + phi)/2, the amount of component C1 */
    double drop_weight;  /* W = sum over phi > 0 of (1 + phi)/2 */
    double drop_count;   /* number of nodes with phi > 0 */
    double centroid[3];  /* sum w x / W over phi > 0, w = (1 + phi)/2 */
    double I[6];         /* central second moments xx yy zz xy xz yz, / W */
    double D;            /* deformation (L - B)/(L + B) of the x-y moment ellipse */
    double theta_deg;    /* inclination of its long axis to x, degrees */
    double p_centre;     /* cs^2 rho + phi mu - (A/4)(phi^2 - 1)^2 at the
                            centroid (trilinear interpolation of the nodes) */
    double p_far;        /* same half a period away in x (and z) */
    double dp;           /* p_centre - p_far (Laplace pressure) */
    double max_u;        /* max |u| */
    long long step;      /* time steps taken since the last initialisation */
    int status;          /* 0 ok, 1 non-finite value seen, 2 |u| > 0.3 */
} fre_obs;

typedef struct fre_ctx fre_ctx;

/* Device bytes a context with these parameters allocates (populations in
 * two buffers, phi/mu fields, geometry, reduction scratch, the component
 * labelling of fre_components); 0 if invalid.  The FP64 staging of the
 * host field and population copies (48 bytes per node, made on their first
 * use) is not included. */
size_t fre_device_bytes(const fre_params *p);

/* Create a context.  cuda_stream is a cudaStream_t (NULL: the context
 * creates its own non-blocking stream).  Validates tau_f, tau_g > 1/2
 * (Eq. bgk, Eq. LBEg), sizes >= 1, nz = 1 for D2Q9, known enums; allocates
 * all device memory with cudaMalloc.  On failure *out is NULL. */
fre_status fre_create(const fre_params *p, void *cuda_stream, fre_ctx **out);

/* Initialise a droplet phi = tanh((R - |x - c|)/(sqrt(2) xi)), xi =
 * sqrt(kappa/A) (model 1: sqrt(2) alpha; the planar profile of Sec. 2.2
 * applied radially), rho = rho0, u = the Couette profile u_x = u_wall (2(y +
 * 1/2)/ny - 1) for the shear device and 0 otherwise, mu from phi, and f =
 * f_eq, g = g_eq (Sec. 2.3).  In 2D cz is ignored.  Needs R > 0 and A > 0,
 * kappa > 0 (model 1: alpha > 0). */
fre_status fre_init_droplet(fre_ctx *c, double cx, double cy, double cz, double R);

/* Initialise from host FP64 fields (n values each; uz may be NULL in 2D):
 * mu from phi, f = f_eq(rho, u), g = g_eq(phi, mu, u).  Values at solid
 * nodes are ignored. */
fre_status fre_init_fields(fre_ctx *c, const double *rho, const double *ux,
                           const double *uy, const double *uz, const double *phi);

/* Consistent initial populations (Sec. 2.3: the populations start at their
 * equilibrium and their kinetic moments are aligned by collisions before the
 * simulated time begins, after Mei et al., Computers & Fluids 2006).  From
 * the current state, which must be freshly initialised or loaded (step 0):
 * take u0 = sum c_i f_i / rho, phi0 = sum g_i, mu0 and the force F0 as they
 * stand; then `iterations` times collide f with the velocity of f_eq and of
 * the forcing term held at u0 and the force at F0 (the density rho = sum f_i
 * is free) and stream it with the walls' rules; finally set g = g_eq(phi0,
 * mu0, u0).  The pressure field, the Laplace pressure of a droplet among
 * it, and the non-equilibrium parts of f then match the initial flow and
 * interface, so the first steps carry no start-up pressure waves.  The step
 * counter stays 0.  Runs on the per-node kernels (any storage format and
 * device) and synchronises; FRE_ERR_STATE if the context has stepped since
 * its initialisation. */
fre_status fre_init_consistent(fre_ctx *c, int iterations);

/* Replace the state by host FP64 pre-collision populations [q][n]; the step
 * counter restarts at 0.  16-bit formats round them to their storage. */
fre_status fre_load_populations(fre_ctx *c, const double *f, const double *g);

/* Copy the pre-collision populations of the current step to host FP64
 * arrays [q][n] (either pointer may be NULL); solid nodes read 0. */
fre_status fre_store_populations(fre_ctx *c, double *f, double *g);

/* Advance nsteps >= 0 time steps; asynchronous on the context stream. */
fre_status fre_step(fre_ctx *c, int nsteps);

/* fre_step with per-kernel device timing: CUDA events are recorded on the
 * context stream before and after each kernel of every step.  ms[0], ms[1],
 * ms[2] receive the summed milliseconds of the phi, mu (including the roller
 * stencil passes) and fused update kernels, ms[3] the whole sequence;
 * launches[0] (if not NULL) the number of kernels launched.  Synchronises. */
fre_status fre_step_timed(fre_ctx *c, int nsteps, double *ms, long long *launches);

/* Macroscopic fields of the current step into host FP64 arrays of n values
 * (any pointer may be NULL); solid nodes read 0.  Synchronises. */
fre_status fre_copy_fields(fre_ctx *c, double *rho, double *ux, double *uy,
                           double *uz, double *phi, double *mu);

/* Observables of the current step (FP64 device reductions); synchronises.
 * Returns FRE_ERR_UNSTABLE (with *out filled) when out->status != 0. */
fre_status fre_observables(fre_ctx *c, fre_obs *out);

/* Connected components of the droplet phase, for breakup detection (Sec. 3:
 * a drop that breaks up leaves separate drops).  The phase is the set of
 * fluid nodes with phi > 0 at the current step (the decision taken in the
 * context's compute precision); two of its nodes are connected when a
 * lattice velocity links them (D2Q9: 8 neighbours, D3Q19: 18), with the
 * device's periodic wrap (x and z always, y except across the shear
 * walls).  *count receives the number of components of at least min_size
 * nodes (min_size <= 1: all); sizes (nullable when max_sizes is 0) the node
 * counts of up to max_sizes of them, largest first, 0 past the last;
 * labels (nullable) n ints: -1 outside the phase, else the smallest node
 * index of the node's component (every component, whatever its size; the
 * labels do not depend on the order of the GPU's threads).  Uses 8 bytes
 * of device memory per node, allocated on the first call and counted by
 * fre_device_bytes.  Synchronises. */
fre_status fre_components(fre_ctx *c, long long min_size, int *count, long long *sizes, int max_sizes, int *labels);

/* Steps taken since the last initialisation. */
long long fre_step_count(const fre_ctx *c);

/* 1 if the time step runs on the row kernels (shared-memory staged x-rows),
 * 0 if on the per-node kernels. */
int fre_uses_row_kernels(const fre_ctx *c);

/* Kernels of the time step: 0 per-node kernels (any geometry and format),
 * 1 warp-specialised kernels on x-chunks, 2 warp-specialised kernels on
 * whole x-rows (FP32 and 16-bit storage, nx up to 512 and a multiple of 64,
 * or of 32 with ny even; the four-roller device stages the wall links of
 * its rollers with the rows and takes its first, in-place step on the
 * per-node kernels); -1 for a NULL context. */
int fre_kernel_path(const fre_ctx *c);

/* Conservation sums and droplet moments without any device allocation.
 *
 * For callers that cannot allocate device memory themselves or let a
 * library do it -- an application whose allocator owns the whole device
 * (a pool carved out at start-up), code running where a cudaMalloc would
 * synchronise or is not allowed -- this computes, from populations the
 * caller owns, what fre_observables reports as mass, phi_sum, volume,
 * drop_weight, drop_count, centroid, I, D and theta_deg.  The paper has no
 * counterpart; it is an interface convenience.
 *
 * f_dev, g_dev: device FP64 pre-collision populations [q][n] in the
 * canonical order (n = nx*ny*nz, x fastest); every node counts as fluid.
 * out_dev: device array of 16 doubles receiving mass, phi_sum, volume,
 * drop_weight, drop_count, centroid[3], I[6] (xx yy zz xy xz yz), D,
 * theta_deg.  cuda_stream: the work is queued there and the call returns
 * without waiting.
 *
 * Scratch: the per-block partial sums live in a static 57,600-byte device
 * array inside the library, which every GPU that loads the library keeps
 * until the process exits.  The first call in a CUDA context (per device,
 * and again after a cudaDeviceReset) looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for that context, so make the first
 * call on each device before any stream capture.  Every call writes all the
 * partials it later reads, so nothing has to start at zero, but all calls
 * share the one array: calls whose work overlaps on the GPU (different
 * streams, or host threads, without ordering between them) race and give
 * wrong results.  No device memory is allocated or freed.  Lattices of more
 * than 2^30 nodes are rejected with FRE_ERR_ARG. */
fre_status fre_moments_noalloc(int lattice, int nx, int ny, int nz, const double *f_dev,
                               const double *g_dev, double *out_dev, void *cuda_stream);

/* ---------------------------------------------------------------- batches
 *
 * A batch holds many independent simulations ("slots") of one lattice and
 * storage format and advances all of them together, for many small or
 * uneven cases (independent droplets, a request stream).  Slots are full
 * contexts created with the batch's stream; a batch step runs either one
 * launch per kernel covering every slot (per-node kernels with a
 * block-to-slot table on the device) or each slot's own fastest kernels;
 * an autotuner times both (and the block width of the first) on the live
 * slot set, and steady steps replay a CUDA graph of two steps.  Every slot
 * computes exactly the update of a context stepped alone; only rounding
 * order may differ between kernel families. */
typedef struct fre_batch fre_batch;

/* Create an empty batch.  budget_bytes bounds the device memory of its
 * slots (fre_device_bytes of each); cuda_stream as in fre_create. */
fre_status fre_batch_create(int lattice, int precision, void *cuda_stream, size_t budget_bytes,
                            fre_batch **out);

/* Admit one case: create a context with *p (its lattice and precision must
 * match the batch) and initialise a droplet as fre_init_droplet does.
 * FRE_ERR_BUDGET (nothing allocated) when it would exceed the budget.
 * *slot receives its slot index (freed slots are reused). */
fre_status fre_batch_add(fre_batch *b, const fre_params *p, double cx, double cy, double cz, double R,
                         int *slot);

/* Finish a slot and free its device memory (synchronises the stream). */
fre_status fre_batch_remove(fre_batch *b, int slot);

/* Advance every slot nsteps steps; asynchronous except for the first call
 * after the slot set changed, which may tune (with real steps). */
fre_status fre_batch_step(fre_batch *b, int nsteps);

/* Observables of one slot (as fre_observables; synchronises). */
fre_status fre_batch_observables(fre_batch *b, int slot, fre_obs *out);

/* The context of a slot (owned by the batch; do not destroy). */
fre_ctx *fre_batch_context(fre_batch *b, int slot);

/* Active slot indices into slots[0..max_slots); returns their number. */
int fre_batch_slots(const fre_batch *b, int *slots, int max_slots);

/* Device bytes held by the slots. */
size_t fre_batch_bytes_in_use(const fre_batch *b);

/* Autotuner result: mode (0 one launch per kernel for all slots, 1 each
 * slot's own kernels one slot after another, 2 each slot's own kernels on
 * four concurrent graph branches), block width, and ms per step measured
 * for the five candidates (batched width 32, 64, 128; per-slot; concurrent)
 * in ms_per_step[0..4].  FRE_ERR_STATE if no
 * tuning is in force: none ran yet, or the slot count has since changed by
 * more than a factor 2 (smaller changes keep the tuned mode). */
fre_status fre_batch_tuning(const fre_batch *b, int *mode, int *bx, double *ms_per_step);

/* Pin the launch mode instead of tuning it: mode 0 (one launch per kernel
 * for all slots, block width bx = 32, 64 or 128), 1 (each slot's own
 * kernels, one slot after another) or 2 (each slot's own kernels on four
 * concurrent graph branches); -1 returns to the autotuner.  Every mode
 * computes the same update of every slot.  Waits for the queued steps;
 * FRE_ERR_ARG for an unknown mode or width.  For tests and for callers that
 * know their best mode. */
fre_status fre_batch_set_mode(fre_batch *b, int mode, int bx);

/* Wait for the batch's queued work. */
fre_status fre_batch_synchronize(fre_batch *b);

/* Destroy the batch and every slot; NULL-safe. */
void fre_batch_destroy(fre_batch *b);

/* ---------------------------------------------------------------- serving
 *
 * A serving loop over a batch: droplet-deformation requests are queued,
 * admitted first come first served under a device-memory budget, advanced
 * together, checked every check_every of their own steps and retired when a
 * stopping rule holds (Sec. 3 measures the deformation D of the droplet):
 *   FRE_SERVE_CONVERGED  |D - D_prev| < tol_D between consecutive checks;
 *   FRE_SERVE_BREAKUP    no node with phi > 0 left, or the phase phi > 0 has
 *                        fallen apart into two or more drops: connected
 *                        components (fre_components) of at least
 *                        breakup_min_frac of the initial droplet's nodes
 *                        (4/3 pi R^3, or pi R^2 in 2D; at least 1);
 *   FRE_SERVE_UNSTABLE   non-finite values or |u| > 0.3;
 *   FRE_SERVE_MAX_STEPS  max_steps reached.
 * Retired contexts stay allocated in a pool and serve later requests of the
 * same geometry (lattice, precision, device, sizes) without allocation; the
 * pool is trimmed when a new geometry needs the budget. */
typedef struct fre_server fre_server;

typedef enum {
    FRE_SERVE_RUNNING = 0,
    FRE_SERVE_CONVERGED = 1,
    FRE_SERVE_BREAKUP = 2,
    FRE_SERVE_MAX_STEPS = 3,
    FRE_SERVE_UNSTABLE = 4,
    FRE_SERVE_REJECTED = 5, /* invalid, or larger than the whole budget */
    FRE_SERVE_FAILED = 6    /* could not be started (e.g. allocation failed) */
} fre_serve_outcome;

typedef struct {
    size_t budget_bytes;     /* device memory of running + pooled contexts */
    long long target_nodes;  /* admit while running nodes stay <= this (0: no limit) */
    int max_running;         /* at most this many running requests (0: no limit) */
    int chunk_steps;         /* steps per fre_server_advance (at most) */
    int check_every;         /* steps of a request between two checks */
    double tol_D;            /* convergence threshold on |D - D_prev| */
    long long max_steps;     /* step cap of a request */
    double breakup_min_frac; /* smallest drop that counts toward a breakup, as a
                                fraction of the initial droplet's nodes, in [0, 1] */
} fre_serve_config;

typedef struct {
    long long id;
    int outcome;        /* fre_serve_outcome */
    long long steps;    /* steps the request ran */
    double t_submit;    /* seconds on the server clock */
    double t_admit;     /* -1 if never admitted */
    double t_done;
    fre_obs obs;        /* observables at the final check (zero if none) */
} fre_serve_result;

typedef struct {
    int running, queued;
    size_t bytes_running, bytes_pooled;
    long long running_nodes;
    long long node_updates;     /* sum over advances of running nodes x steps */
    long long steps_advanced;   /* batch steps issued */
    long long contexts_created, contexts_reused;
    int batch_mode, batch_bx;   /* launch mode in force (see fre_batch_tuning) */
    long long tunes, captures;  /* autotuner runs and graph captures so far */
} fre_serve_stats;

/* Create a server for one lattice and storage format; cuda_stream as in
 * fre_create.  chunk_steps and check_every must be >= 1. */
fre_status fre_server_create(int lattice, int precision, const fre_serve_config *cfg, void *cuda_stream,
                             fre_server **out);

/* Queue a request (parameters, droplet centre and radius); *id receives its
 * id.  A request that can never fit is finished at once as REJECTED (its
 * result is returned by fre_server_results). */
fre_status fre_server_submit(fre_server *s, const fre_params *p, double cx, double cy, double cz, double R,
                             long long *id);

/* Admit what fits (a request's first step, which collides in place, runs
 * on admission: a result's step count includes it), advance every running
 * request by up to chunk_steps
 * steps (stopping early at the next due check), run the due checks and
 * retire finished requests.  *running (nullable) receives the number of
 * requests still running.  Synchronises at each check. */
fre_status fre_server_advance(fre_server *s, int *running);

/* Pop up to max finished results (completion order); returns the count. */
int fre_server_results(fre_server *s, fre_serve_result *out, int max);

fre_status fre_server_stats(const fre_server *s, fre_serve_stats *out);

/* Seconds since fre_server_create (the clock of the result timestamps). */
double fre_server_clock(const fre_server *s);

/* The batch the server advances (owned by the server; do not destroy), e.g.
 * to pin its launch mode with fre_batch_set_mode. */
fre_batch *fre_server_batch(fre_server *s);

/* Destroy the server, its batch and its pool; NULL-safe. */
void fre_server_destroy(fre_server *s);

/* Destroy a context and free its device memory; NULL-safe. */
void fre_destroy(fre_ctx *c);

/* Message of the last failed call on this host thread ("" if none). */
const char *fre_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FRE_H */
