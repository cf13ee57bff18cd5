// Serving loop of the C ABI (include/fre.h, fre_server_*): a request queue
// in front of a batch.  The policy (queue, admission, stopping rules) is the
// host-only ServePolicy; this file is its CUDA executor: it creates or reuses
// contexts, attaches them to the batch, advances the batch and reads the
// observables of the requests whose check is due.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <deque>
#include <map>
#include <vector>

#include "fre_ctx.h"
#include "serve_policy.h"

namespace {

struct Pooled {
    fre_ctx *c;
    size_t bytes;
};

struct Request {
    fre_params p;
    double cx, cy, cz, R;
    fre_ctx *c = nullptr;
    int slot = -1;
    long long min_drop = 1;  // nodes a component needs to count as a drop
    fre_obs last{};
};

fre::ServeLimits limits_of(const fre_serve_config &cfg) {
    fre::ServeLimits l;
    l.budget_bytes = cfg.budget_bytes;
    l.target_nodes = cfg.target_nodes;
    l.max_running = cfg.max_running;
    l.check_every = cfg.check_every;
    l.tol_D = cfg.tol_D;
    l.max_steps = cfg.max_steps;
    return l;
}

fre_status sfail(fre_status s, const char *msg) {
    fre::set_last_error(msg);
    return s;
}

}  // namespace

struct fre_server {
    int lattice = 0, precision = 0, device_id = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fre_serve_config cfg{};
    fre::ServePolicy policy;
    fre_batch *batch = nullptr;
    std::map<long long, Request> req;
    std::vector<Pooled> pool;
    size_t pooled = 0;
    std::deque<fre_serve_result> results;
    std::chrono::steady_clock::time_point t0;
    long long node_updates = 0, steps_advanced = 0, created = 0, reused = 0;

    explicit fre_server(const fre_serve_config &c) : cfg(c), policy(limits_of(c)) {}

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Nodes a connected component of the phase phi > 0 needs to count as a
// drop: breakup_min_frac of the initial droplet's nodes (4/3 pi R^3, or
// pi R^2 in 2D), at least 1.
long long min_drop_nodes(const fre_params &p, double R, double frac) {
    const double pi = 3.14159265358979323846;
    const double v0 = p.lattice == FRE_D3Q19 ? 4.0 / 3.0 * pi * R * R * R : pi * R * R;
    const double m = std::floor(frac * v0);
    return m > 1.0 ? (long long)m : 1;
}

void destroy_pooled(fre_server *s, size_t k) {
    fre_destroy(s->pool[k].c);
    s->pooled -= s->pool[k].bytes;
    s->pool.erase(s->pool.begin() + (long)k);
}

// Hand finished requests to the result queue.
void collect(fre_server *s) {
    for (long long id : s->policy.take_finished()) {
        const fre::ServeJob *j = s->policy.job(id);
        fre_serve_result r{};
        r.id = id;
        r.outcome = j->outcome;
        // plus the first step taken on admission
        r.steps = j->steps + (j->t_admit >= 0.0 && j->outcome != fre::SERVE_FAILED ? 1 : 0);
        r.t_submit = j->t_submit;
        r.t_admit = j->t_admit;
        r.t_done = j->t_done;
        auto it = s->req.find(id);
        if (it != s->req.end()) {
            r.obs = it->second.last;
            s->req.erase(it);
        }
        s->results.push_back(r);
        s->policy.erase(id);
    }
}

// Take a finished request's context out of the batch into the pool.
void retire(fre_server *s, Request &r) {
    if (!r.c) return;
    fre_ctx *c = fre::batch_detach(s->batch, r.slot);
    if (c) {
        const size_t bytes = fre_device_bytes(&c->p);
        s->pool.push_back({c, bytes});
        s->pooled += bytes;
    }
    r.c = nullptr;
    r.slot = -1;
}

// Context for a request: a pooled one of the same geometry, else a new one
// after trimming the pool to the budget left by the running requests.
fre_status start(fre_server *s, long long id) {
    Request &r = s->req[id];
    fre_ctx *c = nullptr;
    const size_t bytes = fre_device_bytes(&r.p);
    for (size_t k = 0; k < s->pool.size(); ++k) {
        if (fre::same_geometry(&s->pool[k].c->p, &r.p)) {
            c = s->pool[k].c;
            s->pooled -= s->pool[k].bytes;
            s->pool.erase(s->pool.begin() + (long)k);
            ++s->reused;
            break;
        }
    }
    fre_status st = FRE_OK;
    if (c) {
        st = fre::ctx_reparam(c, &r.p);
    } else {
        // the policy already counts this request in bytes_in_use
        while (!s->pool.empty() && s->policy.bytes_in_use() + s->pooled > s->cfg.budget_bytes)
            destroy_pooled(s, 0);
        st = fre_create(&r.p, s->stream, &c);
        if (st == FRE_OK) ++s->created;
    }
    if (st == FRE_OK) st = fre_init_droplet(c, r.cx, r.cy, r.cz, r.R);
    // the first step collides in place (no streaming yet); taking it here,
    // on the batch stream, lets the request join the batch's streaming steps
    if (st == FRE_OK) {
        fre::ctx_launch_step(c);
        if (cudaGetLastError() != cudaSuccess) st = sfail(FRE_ERR_CUDA, "fre_server: first step launch failed");
    }
    if (st == FRE_OK) st = fre::batch_attach(s->batch, c, bytes, &r.slot);
    if (st != FRE_OK) {
        if (c) fre_destroy(c);
        r.c = nullptr;
        r.slot = -1;
        return st;
    }
    r.c = c;
    return FRE_OK;
}

}  // namespace

extern "C" {

fre_status fre_server_create(int lattice, int precision, const fre_serve_config *cfg, void *cuda_stream,
                             fre_server **out) {
    if (!out || !cfg) return sfail(FRE_ERR_ARG, "fre_server_create: NULL argument");
    *out = nullptr;
    if (cfg->chunk_steps < 1 || cfg->check_every < 1 || cfg->max_steps < 1 || !(cfg->tol_D >= 0.0) ||
        !(cfg->breakup_min_frac >= 0.0 && cfg->breakup_min_frac <= 1.0))
        return sfail(FRE_ERR_ARG, "fre_server_create: chunk_steps, check_every, max_steps must be >= 1, tol_D >= 0, "
                                  "0 <= breakup_min_frac <= 1");
    fre_server *s = new fre_server(*cfg);
    s->lattice = lattice;
    s->precision = precision;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device_id) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(FRE_ERR_CUDA, "fre_server_create: no CUDA device");
    }
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return sfail(FRE_ERR_CUDA, "fre_server_create: cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    fre_status st = fre_batch_create(lattice, precision, s->stream, cfg->budget_bytes, &s->batch);
    if (st != FRE_OK) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return st;
    }
    *out = s;
    return FRE_OK;
}

fre_status fre_server_submit(fre_server *s, const fre_params *p, double cx, double cy, double cz, double R,
                             long long *id) {
    if (!s || !p || !id) return sfail(FRE_ERR_ARG, "fre_server_submit: NULL argument");
    if (p->lattice != s->lattice || p->precision != s->precision)
        return sfail(FRE_ERR_ARG, "fre_server_submit: lattice and precision must match the server");
    // a request of the full functional (model 1) is rejected: the batch runs model 0
    const size_t bytes = (R > 0.0 && std::isfinite(cx) && std::isfinite(cy) && std::isfinite(cz) && p->model == 0)
                             ? fre_device_bytes(p) : 0;
    const long long nodes = (long long)p->nx * p->ny * p->nz;
    *id = s->policy.submit(nodes, bytes, s->now());
    Request r;
    r.p = *p;
    r.min_drop = bytes ? min_drop_nodes(*p, R, s->cfg.breakup_min_frac) : 1;
    r.cx = cx;
    r.cy = cy;
    r.cz = cz;
    r.R = R;
    s->req[*id] = r;
    collect(s);
    return FRE_OK;
}

fre_status fre_server_advance(fre_server *s, int *running) {
    if (!s) return sfail(FRE_ERR_ARG, "fre_server_advance: server is NULL");
    if (cudaSetDevice(s->device_id) != cudaSuccess) {
        cudaGetLastError();
        return sfail(FRE_ERR_CUDA, "fre_server_advance: cudaSetDevice failed");
    }
    for (long long id : s->policy.admit(s->now())) {
        if (start(s, id) != FRE_OK) s->policy.failed(id, s->now());
    }
    collect(s);
    fre_status st = FRE_OK;
    if (s->policy.running() > 0) {
        long long k = s->policy.steps_to_next_check();
        if (k > s->cfg.chunk_steps) k = s->cfg.chunk_steps;
        st = fre_batch_step(s->batch, (int)k);
        if (st == FRE_OK) {
            s->policy.advanced(k);
            s->node_updates += s->policy.running_nodes() * k;
            s->steps_advanced += k;
            for (long long id : s->policy.due()) {
                Request &r = s->req[id];
                fre_obs o{};
                const fre_status so = fre_observables(r.c, &o);
                if (so != FRE_OK && so != FRE_ERR_UNSTABLE) {
                    s->policy.failed(id, s->now());
                    retire(s, r);
                    continue;
                }
                r.last = o;
                int drops = 0;
                if (o.status == 0 && o.drop_count > 0.0 &&
                    fre_components(r.c, r.min_drop, &drops, nullptr, 0, nullptr) != FRE_OK) {
                    s->policy.failed(id, s->now());
                    retire(s, r);
                    continue;
                }
                const int outcome = s->policy.checked(id, o.D, drops, o.drop_count, o.status, s->now());
                if (outcome != fre::SERVE_RUNNING) retire(s, r);
            }
        }
    }
    collect(s);
    if (running) *running = s->policy.running();
    return st;
}

int fre_server_results(fre_server *s, fre_serve_result *out, int max) {
    if (!s) return -1;
    int n = 0;
    while (n < max && out && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    return n;
}

fre_status fre_server_stats(const fre_server *s, fre_serve_stats *out) {
    if (!s || !out) return sfail(FRE_ERR_ARG, "fre_server_stats: NULL argument");
    out->running = s->policy.running();
    out->queued = s->policy.queued();
    out->bytes_running = s->policy.bytes_in_use();
    out->bytes_pooled = s->pooled;
    out->running_nodes = s->policy.running_nodes();
    out->node_updates = s->node_updates;
    out->steps_advanced = s->steps_advanced;
    out->contexts_created = s->created;
    out->contexts_reused = s->reused;
    fre::batch_counters(s->batch, &out->batch_mode, &out->batch_bx, &out->tunes, &out->captures);
    return FRE_OK;
}

double fre_server_clock(const fre_server *s) { return s ? s->now() : 0.0; }

fre_batch *fre_server_batch(fre_server *s) { return s ? s->batch : nullptr; }

void fre_server_destroy(fre_server *s) {
    if (!s) return;
    cudaSetDevice(s->device_id);
    fre_batch_destroy(s->batch);  // destroys the running contexts
    for (auto &p : s->pool) fre_destroy(p.c);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
