// Internal: the context behind the opaque fre_ctx handle of the C ABI, and
// the pieces of the runtime that the batch runtime reuses.
#pragma once

#include <vector>

#include "fre_internal.h"

struct fre_ctx {
    fre_params p;
    int q = 0;
    int device_id = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    const fre::KernelSet *ks = nullptr;
    fre::Geo G{};
    fre::Phys P{};
    fre::Buf buf[2]{};
    void *phi[2]{};
    void *mu = nullptr;
    void *rhof = nullptr, *murho = nullptr;  // model 1: rho and mu_rho fields
    unsigned char *solid = nullptr;
    int4 *rlinks = nullptr;     // four-roller: the wall links of a plane (Geo::rlinks)
    int4 *rlinkq = nullptr;     // interpolated walls: their fractions (Geo::rlinkq)
    int n_rlinks = 0;
    int *ghost = nullptr;
    int n_ghost = 0;
    double *red = nullptr;
    int red_blocks = 0;
    fre_obs *obs_dev = nullptr;
    fre_obs *obs_host = nullptr;
    int *err_dev = nullptr;  // set by a kernel whose bounded wait timed out
    double *staging = nullptr;
    fre::CclBuffers ccl{};  // component labelling, allocated on first use
    std::vector<void *> allocs;
    int cur = 0;        // buffer holding the state
    int pp = 1;         // phi buffer holding phi of the previous step
    bool local = true;  // state is pre-collision (no streaming pending)
    bool initialised = false;
    bool rows = false;  // the row kernels run the hot path
    int row_w = 0;      // their chunk width
    bool fullrow = false;  // the update runs on the full-row kernel
    long long step = 0;
};

namespace fre {
// launch descriptor of the context's current state
Launch ctx_launch(fre_ctx *c);
// the kernels of one time step on the context stream; advances the state
void ctx_launch_step(fre_ctx *c);
// roller ghost fills of the stencil fields after the phi pass (mu_pass
// false) or the mu pass
void ghost_fields(fre_ctx *c, const Launch &L, bool mu_pass);
// give a context new physical parameters of the same geometry (lattice,
// precision, device, sizes and flags equal); the state must be
// re-initialised before the next step
fre_status ctx_reparam(fre_ctx *c, const fre_params *p);
// true when a context made for *p could serve *q after ctx_reparam
bool same_geometry(const fre_params *p, const fre_params *q);
}  // namespace fre

struct fre_batch;
namespace fre {
// hand an existing context (created on the batch stream, initialised) to a
// batch as a new slot; `bytes` is charged to the batch budget
fre_status batch_attach(fre_batch *b, fre_ctx *c, size_t bytes, int *slot);
// take a slot's context out of a batch without synchronising or freeing it
// (work already queued on the stream still uses it)
fre_ctx *batch_detach(fre_batch *b, int slot);
// the stream of a batch
cudaStream_t batch_stream(const fre_batch *b);
// launch mode in force and the counts of autotuner runs and graph captures
void batch_counters(const fre_batch *b, int *mode, int *bx, long long *tunes, long long *captures);
}  // namespace fre
