// Test-only C wrapper of the host serving policy (ServePolicy) so the host
// tests can drive it with a fake executor; built by the tests with g++.
#include <vector>

#include "serve_policy.h"

extern "C" {

void *sp_create(unsigned long long budget, long long target_nodes, int max_running, int check_every, double tol_D,
                long long max_steps) {
    fre::ServeLimits l;
    l.budget_bytes = (size_t)budget;
    l.target_nodes = target_nodes;
    l.max_running = max_running;
    l.check_every = check_every;
    l.tol_D = tol_D;
    l.max_steps = max_steps;
    return new fre::ServePolicy(l);
}

void sp_destroy(void *p) { delete static_cast<fre::ServePolicy *>(p); }

long long sp_submit(void *p, long long nodes, unsigned long long bytes, double t) {
    return static_cast<fre::ServePolicy *>(p)->submit(nodes, (size_t)bytes, t);
}

static int copy_ids(const std::vector<long long> &v, long long *out, int max) {
    int n = 0;
    for (long long id : v)
        if (n < max) out[n++] = id;
    return (int)v.size();
}

int sp_admit(void *p, double t, long long *out, int max) {
    return copy_ids(static_cast<fre::ServePolicy *>(p)->admit(t), out, max);
}

void sp_failed(void *p, long long id, double t) { static_cast<fre::ServePolicy *>(p)->failed(id, t); }

void sp_advanced(void *p, long long steps) { static_cast<fre::ServePolicy *>(p)->advanced(steps); }

int sp_due(void *p, long long *out, int max) { return copy_ids(static_cast<fre::ServePolicy *>(p)->due(), out, max); }

long long sp_steps_to_next_check(void *p) { return static_cast<fre::ServePolicy *>(p)->steps_to_next_check(); }

int sp_checked(void *p, long long id, double D, int components, double count, int status, double t) {
    return static_cast<fre::ServePolicy *>(p)->checked(id, D, components, count, status, t);
}

int sp_take_finished(void *p, long long *out, int max) {
    return copy_ids(static_cast<fre::ServePolicy *>(p)->take_finished(), out, max);
}

// outcome, steps, t_admit, t_done of a job; returns 0 if unknown
int sp_job(void *p, long long id, int *outcome, long long *steps, double *t_admit, double *t_done) {
    const fre::ServeJob *j = static_cast<fre::ServePolicy *>(p)->job(id);
    if (!j) return 0;
    *outcome = j->outcome;
    *steps = j->steps;
    *t_admit = j->t_admit;
    *t_done = j->t_done;
    return 1;
}

int sp_running(void *p) { return static_cast<fre::ServePolicy *>(p)->running(); }
int sp_queued(void *p) { return static_cast<fre::ServePolicy *>(p)->queued(); }
unsigned long long sp_bytes(void *p) { return static_cast<fre::ServePolicy *>(p)->bytes_in_use(); }
long long sp_running_nodes(void *p) { return static_cast<fre::ServePolicy *>(p)->running_nodes(); }

}  // extern "C"
