// Host-side policy of the serving loop (C ABI fre_server_*): the request
// queue, admission under a device-memory budget, per-request step counting,
// and the stopping rules of a droplet-deformation run.  Plain C++17 with no
// CUDA dependency, so the same code runs under the CUDA executor and under a
// fake executor in the host tests.
//
// Stopping rules (checked every `check_every` steps of a request):
//   converged -- |D - D_prev| < tol_D between two consecutive checks, D the
//                deformation of the droplet's moment ellipse (Sec. 3);
//   breakup   -- no node with phi > 0 is left, or the phase phi > 0 falls
//                apart into two or more connected components (the drop
//                split; the executor counts the components large enough to
//                be drops, fre_components);
//   unstable  -- the observables saw non-finite values or |u| > 0.3;
//   max_steps -- the request reached its step cap.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace fre {

enum ServeOutcome {
    SERVE_RUNNING = 0,
    SERVE_CONVERGED = 1,
    SERVE_BREAKUP = 2,
    SERVE_MAX_STEPS = 3,
    SERVE_UNSTABLE = 4,
    SERVE_REJECTED = 5,  // larger than the whole budget, or invalid
    SERVE_FAILED = 6,    // the executor could not start or advance it
};

struct ServeLimits {
    size_t budget_bytes = 0;     // device memory of all running requests
    long long target_nodes = 0;  // admit while running nodes < target (0: no limit)
    int max_running = 0;         // at most this many running (0: no limit)
    int check_every = 1000;      // steps between two checks of a request
    double tol_D = 1e-4;         // convergence threshold on |D - D_prev|
    long long max_steps = 100000;
};

struct ServeJob {
    long long id = 0;
    long long nodes = 0;
    size_t bytes = 0;
    double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
    long long steps = 0;      // steps taken since admission
    long long next_check = 0;  // step count of its next check
    int checks = 0;
    double D_prev = 0.0, D = 0.0;
    int components = 0;  // drops found at the last check
    int outcome = SERVE_RUNNING;
    bool running = false;
};

class ServePolicy {
  public:
    explicit ServePolicy(const ServeLimits &lim) : lim_(lim) {
        if (lim_.check_every < 1) lim_.check_every = 1;
    }

    const ServeLimits &limits() const { return lim_; }

    // Queue a request; returns its id.  A request that can never fit the
    // budget is finished at once as REJECTED.
    long long submit(long long nodes, size_t bytes, double t_now) {
        ServeJob j;
        j.id = next_id_++;
        j.nodes = nodes;
        j.bytes = bytes;
        j.t_submit = t_now;
        jobs_[j.id] = j;
        if (bytes == 0 || bytes > lim_.budget_bytes) {
            finish(jobs_[j.id], SERVE_REJECTED, t_now);
        } else {
            queue_.push_back(j.id);
        }
        return j.id;
    }

    // Requests to start now, first come first served: the head of the queue
    // starts while it fits the budget and the running limits (the first one
    // always starts on an idle server).  Their bytes are reserved.
    std::vector<long long> admit(double t_now) {
        std::vector<long long> out;
        while (!queue_.empty()) {
            ServeJob &j = jobs_[queue_.front()];
            if (in_use_ + j.bytes > lim_.budget_bytes) break;
            if (n_running_ > 0) {
                if (lim_.max_running > 0 && n_running_ >= lim_.max_running) break;
                if (lim_.target_nodes > 0 && running_nodes_ + j.nodes > lim_.target_nodes) break;
            }
            queue_.pop_front();
            j.running = true;
            j.t_admit = t_now;
            j.steps = 0;
            j.next_check = lim_.check_every;
            in_use_ += j.bytes;
            running_nodes_ += j.nodes;
            ++n_running_;
            out.push_back(j.id);
        }
        return out;
    }

    // The executor could not start or advance a running request.
    void failed(long long id, double t_now) {
        auto it = jobs_.find(id);
        if (it == jobs_.end() || it->second.outcome != SERVE_RUNNING) return;
        finish(it->second, SERVE_FAILED, t_now);
    }

    // Every running request advanced by `steps`.
    void advanced(long long steps) {
        for (auto &kv : jobs_)
            if (kv.second.running) kv.second.steps += steps;
    }

    // Running requests whose check is due (steps reached next_check or the cap).
    std::vector<long long> due() const {
        std::vector<long long> out;
        for (const auto &kv : jobs_) {
            const ServeJob &j = kv.second;
            if (j.running && (j.steps >= j.next_check || j.steps >= lim_.max_steps)) out.push_back(j.id);
        }
        return out;
    }

    // Steps until the earliest due check or cap among running requests
    // (0 when nothing runs).
    long long steps_to_next_check() const {
        long long best = 0;
        for (const auto &kv : jobs_) {
            const ServeJob &j = kv.second;
            if (!j.running) continue;
            long long s = j.next_check - j.steps;
            const long long cap = lim_.max_steps - j.steps;
            if (cap < s) s = cap;
            if (s < 1) s = 1;
            if (best == 0 || s < best) best = s;
        }
        return best;
    }

    // Result of a check: D, the number of drops (connected components of
    // the phase phi > 0 large enough to count), the nodes with phi > 0, and
    // the observables status (0 ok).  Returns the outcome (RUNNING to go on).
    int checked(long long id, double D, int components, double drop_count, int status, double t_now) {
        auto it = jobs_.find(id);
        if (it == jobs_.end() || !it->second.running) return SERVE_FAILED;
        ServeJob &j = it->second;
        j.D_prev = j.D;
        j.D = D;
        j.components = components;
        ++j.checks;
        j.next_check = j.steps + lim_.check_every;
        int out = SERVE_RUNNING;
        if (status != 0) out = SERVE_UNSTABLE;
        else if (drop_count <= 0.0 || components >= 2) out = SERVE_BREAKUP;
        else if (j.checks >= 2 && (j.D - j.D_prev < lim_.tol_D && j.D_prev - j.D < lim_.tol_D)) out = SERVE_CONVERGED;
        else if (j.steps >= lim_.max_steps) out = SERVE_MAX_STEPS;
        if (out != SERVE_RUNNING) finish(j, out, t_now);
        return out;
    }

    // Finished requests not yet handed out, in completion order.
    std::vector<long long> take_finished() {
        std::vector<long long> out(finished_.begin(), finished_.end());
        finished_.clear();
        return out;
    }

    const ServeJob *job(long long id) const {
        auto it = jobs_.find(id);
        return it == jobs_.end() ? nullptr : &it->second;
    }

    // Forget a finished request once its result has been handed out.
    void erase(long long id) {
        auto it = jobs_.find(id);
        if (it != jobs_.end() && !it->second.running) jobs_.erase(it);
    }

    int running() const { return n_running_; }
    int queued() const { return (int)queue_.size(); }
    size_t bytes_in_use() const { return in_use_; }
    long long running_nodes() const { return running_nodes_; }

  private:
    void finish(ServeJob &j, int outcome, double t_now) {
        if (j.running) {
            in_use_ -= j.bytes;
            running_nodes_ -= j.nodes;
            --n_running_;
            j.running = false;
        } else {
            for (auto it = queue_.begin(); it != queue_.end(); ++it)
                if (*it == j.id) {
                    queue_.erase(it);
                    break;
                }
        }
        j.outcome = outcome;
        j.t_done = t_now;
        finished_.push_back(j.id);
    }

    ServeLimits lim_;
    std::map<long long, ServeJob> jobs_;
    std::deque<long long> queue_;
    std::deque<long long> finished_;
    long long next_id_ = 1;
    size_t in_use_ = 0;
    long long running_nodes_ = 0;
    int n_running_ = 0;
};

}  // namespace fre
