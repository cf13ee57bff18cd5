// Batch runtime of the C ABI (include/fre.h, fre_batch_*): many independent
// simulations ("slots") of one lattice and storage format on one stream.
//
// A batch step advances every active slot.  Two execution modes:
//   batched   -- one launch per kernel for all slots (per-node kernels,
//                block -> slot table on the device; block width BX tuned);
//   per-slot  -- each slot's own fastest kernels, back to back.
// The autotuner times the candidates on the live slot set (the timed steps
// are real steps) and keeps the fastest.  Steady-state steps replay a CUDA
// graph of two consecutive steps (even and odd buffer parity), so the host
// cost of a step does not grow with the number of slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "fre_ctx.h"

struct fre_batch {
    int lattice = 0, precision = 0;
    int device_id = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, in_use = 0;
    std::vector<fre_ctx *> slots;
    std::vector<size_t> slot_bytes;
    const fre::BatchKernels *bk = nullptr;
    // device tables of the batched mode
    fre::Launch *d_cases[2] = {nullptr, nullptr};
    int *d_bstart = nullptr, *d_gstart = nullptr;
    int cap = 0;
    std::vector<int> order;  // active slots, table order
    bool tables_valid = false;
    int table_bx = 0;  // block width the block prefix was built for
    int total_blocks = 0, total_ghost_blocks = 0;
    // tuning and graph
    int mode = 0;  // 0 batched, 1 per-slot, 2 per-slot on concurrent streams
    int bx = 64;
    bool tuned = false;
    bool pinned = false;   // mode fixed by fre_batch_set_mode: no tuning
    int tuned_nslots = 0;  // slot count the tuning was measured on
    double tuned_ms[5] = {0, 0, 0, 0, 0};  // ms/step of batched bx 32, 64, 128, per-slot, concurrent
    // streams and events of the concurrent mode (graph branches)
    static constexpr int kBranches = 16;
    cudaStream_t aux[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaGraphExec_t graph = nullptr;
    long long graph_replays = 0;
    long long n_tunes = 0, n_captures = 0;
};

namespace {

fre_status bfail(fre_status s, const char *fmt, const char *detail = "") {
    char msg[512];
    snprintf(msg, sizeof(msg), fmt, detail);
    fre::set_last_error(msg);
    return s;
}

#define BCUDA(call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return bfail(FRE_ERR_CUDA, #call ": %s", cudaGetErrorString(e_)); \
    } while (0)

void drop_graph(fre_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

std::vector<int> active(const fre_batch *b) {
    std::vector<int> a;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (b->slots[i]) a.push_back(i);
    return a;
}

// The slot set changed: tables and graph are rebuilt; the tuned launch mode
// is kept while the slot count stays within a factor 2 of the tuned one.
void invalidate(fre_batch *b) {
    b->tables_valid = false;
    drop_graph(b);
    if (b->tuned && !b->pinned) {
        const int n = (int)active(b).size();
        if (2 * n < b->tuned_nslots || n > 2 * b->tuned_nslots) b->tuned = false;
    }
}

// launch descriptor of a context after one more step (buffers swapped)
fre::Launch next_launch(fre_ctx *c) {
    c->cur ^= 1;
    c->pp ^= 1;
    fre::Launch L = fre::ctx_launch(c);
    c->cur ^= 1;
    c->pp ^= 1;
    L.pull = 1;
    return L;
}

fre_status build_tables(fre_batch *b) {
    b->order = active(b);
    const int n = (int)b->order.size();
    if (n > b->cap) {
        for (auto &p : b->d_cases) {
            if (p) cudaFree(p);
            p = nullptr;
        }
        if (b->d_bstart) cudaFree(b->d_bstart);
        if (b->d_gstart) cudaFree(b->d_gstart);
        b->d_bstart = b->d_gstart = nullptr;
        const int cap = std::max(64, n * 2);
        BCUDA(cudaMalloc(&b->d_cases[0], sizeof(fre::Launch) * cap));
        BCUDA(cudaMalloc(&b->d_cases[1], sizeof(fre::Launch) * cap));
        BCUDA(cudaMalloc(&b->d_bstart, sizeof(int) * (cap + 1)));
        BCUDA(cudaMalloc(&b->d_gstart, sizeof(int) * (cap + 1)));
        b->cap = cap;
    }
    std::vector<fre::Launch> A(n), B(n);
    std::vector<int> gs(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        fre_ctx *c = b->slots[b->order[k]];
        A[k] = fre::ctx_launch(c);
        A[k].pull = c->local ? 0 : 1;
        B[k] = next_launch(c);
        gs[k + 1] = gs[k] + (c->n_ghost + 255) / 256;
    }
    b->total_ghost_blocks = gs[n];
    b->table_bx = 0;  // the block prefix follows the slot order
    BCUDA(cudaMemcpyAsync(b->d_cases[0], A.data(), sizeof(fre::Launch) * n, cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaMemcpyAsync(b->d_cases[1], B.data(), sizeof(fre::Launch) * n, cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaMemcpyAsync(b->d_gstart, gs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    b->tables_valid = true;
    return FRE_OK;
}

// block prefix of the batched kernels for block width bx
fre_status upload_blocks(fre_batch *b, int bx) {
    const int n = (int)b->order.size();
    const int by = 256 / bx;
    std::vector<int> bs(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        const fre_ctx *c = b->slots[b->order[k]];
        const long long nb = (long long)((c->p.nx + bx - 1) / bx) * ((c->p.ny + by - 1) / by) * c->p.nz;
        if (bs[k] + nb > (1LL << 31) - 1) return bfail(FRE_ERR_ARG, "fre_batch: too many blocks%s");
        bs[k + 1] = bs[k] + (int)nb;
    }
    b->total_blocks = bs[n];
    BCUDA(cudaMemcpyAsync(b->d_bstart, bs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    b->table_bx = bx;
    return FRE_OK;
}

fre::BatchLaunch batch_launch(fre_batch *b, int which) {
    fre::BatchLaunch B{};
    B.cases = b->d_cases[which];
    B.block_start = b->d_bstart;
    B.ghost_start = b->d_gstart;
    B.nslots = (int)b->order.size();
    B.total_blocks = b->total_blocks;
    B.total_ghost_blocks = b->total_ghost_blocks;
    B.stream = b->stream;
    return B;
}

// kernels of one step of every slot in batched mode, descriptors `which`
void launch_batched(fre_batch *b, int which) {
    const fre::BatchLaunch B = batch_launch(b, which);
    b->bk->phi(B, b->bx);
    if (B.total_ghost_blocks) b->bk->ghost(B, 0);
    b->bk->mu(B, b->bx);
    if (B.total_ghost_blocks) b->bk->ghost(B, 1);
    b->bk->update(B, b->bx);
}

// advance the host state of every slot by one step (after batched kernels)
void advance_state(fre_batch *b) {
    for (int s : b->order) {
        fre_ctx *c = b->slots[s];
        c->cur ^= 1;
        c->pp ^= 1;
        c->local = false;
        c->step++;
    }
}

// one step outside any graph
fre_status single_step(fre_batch *b) {
    if (b->mode == 0) {
        if (!b->tables_valid) {
            fre_status s = build_tables(b);
            if (s != FRE_OK) return s;
            b->table_bx = 0;
        }
        if (b->table_bx != b->bx) {
            fre_status s = upload_blocks(b, b->bx);
            if (s != FRE_OK) return s;
        }
        launch_batched(b, 0);
        const bool had_local = [&] {
            for (int s : b->order)
                if (b->slots[s]->local) return true;
            return false;
        }();
        advance_state(b);
        // descriptors A and B swap roles; a slot that streamed in place
        // changes its pull flag, which needs a rebuild
        if (had_local) {
            b->tables_valid = false;
        } else {
            std::swap(b->d_cases[0], b->d_cases[1]);
        }
        drop_graph(b);
    } else {
        // per-slot modes: one slot after another outside a graph
        b->order = active(b);
        for (int s : b->order) fre::ctx_launch_step(b->slots[s]);
        b->tables_valid = false;  // buffer parities changed
        drop_graph(b);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(FRE_ERR_CUDA, "fre_batch_step: %s", cudaGetErrorString(e));
    return FRE_OK;
}

// capture the two-step graph of the current mode
fre_status capture(fre_batch *b) {
    drop_graph(b);
    if (b->mode == 0) {
        if (!b->tables_valid) {
            fre_status s = build_tables(b);
            if (s != FRE_OK) return s;
            b->table_bx = 0;
        }
        if (b->table_bx != b->bx) {
            fre_status s = upload_blocks(b, b->bx);
            if (s != FRE_OK) return s;
        }
    } else {
        b->order = active(b);
    }
    ++b->n_captures;
    if (b->mode == 2 && !b->fork) {
        // streams and events of the graph branches, made once
        BCUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (int j = 0; j < fre_batch::kBranches; ++j) {
            BCUDA(cudaStreamCreateWithFlags(&b->aux[j], cudaStreamNonBlocking));
            BCUDA(cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming));
        }
    }
    BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (b->mode == 0) {
        launch_batched(b, 0);
        launch_batched(b, 1);
    } else if (b->mode == 1) {
        for (int s : b->order) fre::ctx_launch_step(b->slots[s]);
        for (int s : b->order) fre::ctx_launch_step(b->slots[s]);
        for (int s : b->order) b->slots[s]->step -= 2;  // captured, not run
    } else {
        // each slot's two steps on one branch, so that the slots' kernels
        // may run side by side; the largest slots first, each onto the
        // branch with the fewest nodes so far, so that the branches end
        // together
        cudaEventRecord(b->fork, b->stream);
        for (int j = 0; j < fre_batch::kBranches; ++j) cudaStreamWaitEvent(b->aux[j], b->fork, 0);
        auto nodes = [&](int s) { return (long long)b->slots[s]->G.nx * b->slots[s]->G.ny * b->slots[s]->G.nz; };
        std::vector<int> by_size(b->order);
        std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) { return nodes(x) > nodes(y); });
        long long load[fre_batch::kBranches] = {};
        for (int s : by_size) {
            fre_ctx *c = b->slots[s];
            const cudaStream_t own = c->stream;
            int j = 0;
            for (int q = 1; q < fre_batch::kBranches; ++q)
                if (load[q] < load[j]) j = q;
            load[j] += nodes(s);
            c->stream = b->aux[j];
            fre::ctx_launch_step(c);
            fre::ctx_launch_step(c);
            c->stream = own;
            c->step -= 2;  // captured, not run
        }
        for (int j = 0; j < fre_batch::kBranches; ++j) {
            cudaEventRecord(b->join[j], b->aux[j]);
            cudaStreamWaitEvent(b->stream, b->join[j], 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(FRE_ERR_CUDA, "fre_batch: graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bfail(FRE_ERR_CUDA, "fre_batch: graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return FRE_OK;
}

fre_status replay(fre_batch *b, long long pairs) {
    for (long long k = 0; k < pairs; ++k) BCUDA(cudaGraphLaunch(b->graph, b->stream));
    for (int s : b->order) b->slots[s]->step += 2 * pairs;
    b->graph_replays += pairs;
    return FRE_OK;
}

bool any_local(const fre_batch *b) {
    for (auto *c : b->slots)
        if (c && c->local) return true;
    return false;
}

// Time the candidates on the live slot set: each takes one plain step (so
// every kernel it uses has run once outside a capture), is captured, and
// runs 3 graph replays, the last 2 timed -- 7 real steps per candidate.
constexpr int kTuneSteps = 35;
fre_status autotune(fre_batch *b, long long *taken) {
    ++b->n_tunes;
    const int modes[5] = {0, 0, 0, 1, 2};
    const int bxs[5] = {32, 64, 128, 64, 64};
    double best = 1e300;
    int best_k = 1;
    // the two timing events, destroyed on every way out of the loop
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
            for (auto ev : e)
                if (ev) cudaEventDestroy(ev);
        }
    } ev;
    BCUDA(cudaEventCreate(&ev.e[0]));
    BCUDA(cudaEventCreate(&ev.e[1]));
    const cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    for (int k = 0; k < 5; ++k) {
        b->mode = modes[k];
        b->bx = bxs[k];
        fre_status s = single_step(b);
        if (s != FRE_OK) return s;
        *taken += 1;
        s = capture(b);
        if (s != FRE_OK) return s;
        s = replay(b, 1);  // warm-up
        if (s != FRE_OK) return s;
        cudaEventRecord(e0, b->stream);
        s = replay(b, 2);
        if (s != FRE_OK) return s;
        cudaEventRecord(e1, b->stream);
        BCUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->tuned_ms[k] = ms / 4.0;
        *taken += 6;
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    b->mode = modes[best_k];
    b->bx = bxs[best_k];
    b->tuned = true;
    b->tuned_nslots = (int)active(b).size();
    return capture(b);
}

fre_status benter(fre_batch *b) {
    if (!b) return bfail(FRE_ERR_ARG, "batch is NULL%s");
    BCUDA(cudaSetDevice(b->device_id));
    return FRE_OK;
}

}  // namespace

fre_status fre::batch_attach(fre_batch *b, fre_ctx *c, size_t bytes, int *slot) {
    if (!b || !c || !slot) return bfail(FRE_ERR_ARG, "batch_attach: NULL argument%s");
    if (c->p.lattice != b->lattice || c->p.precision != b->precision || c->stream != b->stream)
        return bfail(FRE_ERR_ARG, "batch_attach: lattice, precision and stream must match the batch%s");
    if (!c->initialised) return bfail(FRE_ERR_STATE, "batch_attach: context not initialised%s");
    if (c->p.model != 0) return bfail(FRE_ERR_ARG, "batch_attach: batches run the reduced functional (model 0)%s");
    if (c->p.flags & FRE_FLAG_INTERPOLATED_WALLS)
        return bfail(FRE_ERR_ARG, "batch_attach: batches run half-way bounce-back at the rollers%s");
    if (b->in_use + bytes > b->budget) return bfail(FRE_ERR_BUDGET, "batch_attach: device-memory budget exceeded%s");
    int k = 0;
    while (k < (int)b->slots.size() && b->slots[k]) ++k;
    if (k == (int)b->slots.size()) {
        b->slots.push_back(nullptr);
        b->slot_bytes.push_back(0);
    }
    b->slots[k] = c;
    b->slot_bytes[k] = bytes;
    b->in_use += bytes;
    *slot = k;
    invalidate(b);
    return FRE_OK;
}

fre_ctx *fre::batch_detach(fre_batch *b, int slot) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot]) return nullptr;
    fre_ctx *c = b->slots[slot];
    b->slots[slot] = nullptr;
    b->in_use -= b->slot_bytes[slot];
    b->slot_bytes[slot] = 0;
    invalidate(b);
    return c;
}

cudaStream_t fre::batch_stream(const fre_batch *b) { return b ? b->stream : nullptr; }

void fre::batch_counters(const fre_batch *b, int *mode, int *bx, long long *tunes, long long *captures) {
    *mode = b->mode;
    *bx = b->bx;
    *tunes = b->n_tunes;
    *captures = b->n_captures;
}

extern "C" {

fre_status fre_batch_create(int lattice, int precision, void *cuda_stream, size_t budget_bytes, fre_batch **out) {
    if (!out) return bfail(FRE_ERR_ARG, "fre_batch_create: out is NULL%s");
    *out = nullptr;
    if (lattice != FRE_D2Q9 && lattice != FRE_D3Q19) return bfail(FRE_ERR_ARG, "fre_batch_create: unknown lattice%s");
    if (precision < FRE_FP64 || precision > FRE_BF16DEV)
        return bfail(FRE_ERR_ARG, "fre_batch_create: unknown precision%s");
    fre_batch *b = new fre_batch();
    b->lattice = lattice;
    b->precision = precision;
    b->budget = budget_bytes;
    b->bk = lattice == FRE_D2Q9 ? fre::batch_kernels_d2q9(precision) : fre::batch_kernels_d3q19(precision);
    if (cudaGetDevice(&b->device_id) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(FRE_ERR_CUDA, "fre_batch_create: no CUDA device%s");
    }
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(FRE_ERR_CUDA, "fre_batch_create: cudaStreamCreate failed%s");
        }
        b->own_stream = true;
    }
    *out = b;
    return FRE_OK;
}

fre_status fre_batch_add(fre_batch *b, const fre_params *p, double cx, double cy, double cz, double R, int *slot) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    if (!p || !slot) return bfail(FRE_ERR_ARG, "fre_batch_add: NULL argument%s");
    if (p->lattice != b->lattice || p->precision != b->precision)
        return bfail(FRE_ERR_ARG, "fre_batch_add: lattice and precision must match the batch%s");
    if (p->model != 0) return bfail(FRE_ERR_ARG, "fre_batch_add: batches run the reduced functional (model 0)%s");
    if (p->flags & FRE_FLAG_INTERPOLATED_WALLS)
        return bfail(FRE_ERR_ARG, "fre_batch_add: batches run half-way bounce-back at the rollers%s");
    const size_t bytes = fre_device_bytes(p);
    if (bytes == 0) return bfail(FRE_ERR_ARG, "fre_batch_add: invalid parameters%s");
    if (b->in_use + bytes > b->budget) return bfail(FRE_ERR_BUDGET, "fre_batch_add: device-memory budget exceeded%s");
    fre_ctx *c = nullptr;
    s = fre_create(p, b->stream, &c);
    if (s != FRE_OK) return s;
    s = fre_init_droplet(c, cx, cy, cz, R);
    if (s != FRE_OK) {
        fre_destroy(c);
        return s;
    }
    int k = 0;
    while (k < (int)b->slots.size() && b->slots[k]) ++k;
    if (k == (int)b->slots.size()) {
        b->slots.push_back(nullptr);
        b->slot_bytes.push_back(0);
    }
    b->slots[k] = c;
    b->slot_bytes[k] = bytes;
    b->in_use += bytes;
    *slot = k;
    invalidate(b);
    return FRE_OK;
}

fre_status fre_batch_remove(fre_batch *b, int slot) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
        return bfail(FRE_ERR_ARG, "fre_batch_remove: no such slot%s");
    BCUDA(cudaStreamSynchronize(b->stream));
    fre_destroy(b->slots[slot]);
    b->slots[slot] = nullptr;
    b->in_use -= b->slot_bytes[slot];
    b->slot_bytes[slot] = 0;
    invalidate(b);
    return FRE_OK;
}

fre_status fre_batch_step(fre_batch *b, int nsteps) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    if (nsteps < 0) return bfail(FRE_ERR_ARG, "fre_batch_step: nsteps < 0%s");
    if (active(b).empty() || nsteps == 0) return FRE_OK;
    long long left = nsteps;
    // slots that still hold in-place populations take one batched step first
    if (any_local(b)) {
        const int m = b->mode;
        b->mode = 0;
        s = single_step(b);
        b->mode = m;
        if (s != FRE_OK) return s;
        --left;
    }
    if (!b->tuned && left >= kTuneSteps + 4) {
        long long taken = 0;
        s = autotune(b, &taken);
        if (s != FRE_OK) return s;
        left -= taken;
    }
    if (left >= 2) {
        if (!b->graph) {
            s = capture(b);
            if (s != FRE_OK) return s;
        }
        s = replay(b, left / 2);
        if (s != FRE_OK) return s;
        left -= 2 * (left / 2);
    }
    if (left == 1) {
        s = single_step(b);
        if (s != FRE_OK) return s;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(FRE_ERR_CUDA, "fre_batch_step: %s", cudaGetErrorString(e));
    return FRE_OK;
}

fre_status fre_batch_observables(fre_batch *b, int slot, fre_obs *out) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
        return bfail(FRE_ERR_ARG, "fre_batch_observables: no such slot%s");
    return fre_observables(b->slots[slot], out);
}

fre_ctx *fre_batch_context(fre_batch *b, int slot) {
    if (!b || slot < 0 || slot >= (int)b->slots.size()) return nullptr;
    return b->slots[slot];
}

int fre_batch_slots(const fre_batch *b, int *slots, int max_slots) {
    if (!b) return -1;
    int n = 0;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (b->slots[i]) {
            if (slots && n < max_slots) slots[n] = i;
            ++n;
        }
    return n;
}

size_t fre_batch_bytes_in_use(const fre_batch *b) { return b ? b->in_use : 0; }

fre_status fre_batch_tuning(const fre_batch *b, int *mode, int *bx, double *ms_per_step) {
    if (!b) return bfail(FRE_ERR_ARG, "batch is NULL%s");
    if (mode) *mode = b->mode;
    if (bx) *bx = b->bx;
    if (ms_per_step)
        for (int k = 0; k < 5; ++k) ms_per_step[k] = b->tuned_ms[k];
    return b->tuned ? FRE_OK : FRE_ERR_STATE;
}

fre_status fre_batch_set_mode(fre_batch *b, int mode, int bx) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    if (mode < -1 || mode > 2) return bfail(FRE_ERR_ARG, "fre_batch_set_mode: mode must be -1, 0, 1 or 2%s");
    if (mode == 0 && bx != 32 && bx != 64 && bx != 128)
        return bfail(FRE_ERR_ARG, "fre_batch_set_mode: bx must be 32, 64 or 128%s");
    // queued steps of the old mode finish first; the next step captures anew
    BCUDA(cudaStreamSynchronize(b->stream));
    drop_graph(b);
    b->tables_valid = false;
    if (mode < 0) {
        b->pinned = false;
        b->tuned = false;
        return FRE_OK;
    }
    b->pinned = true;
    b->tuned = true;
    b->mode = mode;
    b->bx = mode == 0 ? bx : 64;
    b->tuned_nslots = (int)active(b).size();
    for (double &m : b->tuned_ms) m = 0.0;
    return FRE_OK;
}

fre_status fre_batch_synchronize(fre_batch *b) {
    fre_status s = benter(b);
    if (s != FRE_OK) return s;
    BCUDA(cudaStreamSynchronize(b->stream));
    return FRE_OK;
}

void fre_batch_destroy(fre_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device_id);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto *c : b->slots)
        if (c) fre_destroy(c);
    for (auto *p : b->d_cases)
        if (p) cudaFree(p);
    if (b->d_bstart) cudaFree(b->d_bstart);
    if (b->d_gstart) cudaFree(b->d_gstart);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    if (b->fork) {
        cudaEventDestroy(b->fork);
        for (int j = 0; j < fre_batch::kBranches; ++j) {
            cudaStreamDestroy(b->aux[j]);
            cudaEventDestroy(b->join[j]);
        }
    }
    cudaGetLastError();
    delete b;
}

}  // extern "C"
