"""The host policy of the serving loop (csrc/serve_policy.h), driven on the CPU
through a test-only C wrapper and a fake executor: FIFO admission under the
device-memory budget and the running limits, the stopping rules (converged,
breakup, unstable, step cap), and failures injected on the host (an executor
that cannot start a request, or loses one while it runs)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_01617_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "native", "serve_policy_shim.cpp")

RUNNING, CONVERGED, BREAKUP, MAX_STEPS, UNSTABLE, REJECTED, FAILED = range(7)


@pytest.fixture(scope="module")
def sp(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("shim") / "libserve_policy_shim.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, SHIM, "-o", out], check=True)
    L = C.CDLL(out)
    vp, ll, d = C.c_void_p, C.c_longlong, C.c_double
    L.sp_create.restype = vp
    L.sp_create.argtypes = [C.c_ulonglong, ll, C.c_int, C.c_int, d, ll]
    L.sp_destroy.argtypes = [vp]
    L.sp_submit.restype = ll
    L.sp_submit.argtypes = [vp, ll, C.c_ulonglong, d]
    for name in ("sp_admit", "sp_due", "sp_take_finished"):
        getattr(L, name).restype = C.c_int
    L.sp_admit.argtypes = [vp, d, C.POINTER(ll), C.c_int]
    L.sp_due.argtypes = [vp, C.POINTER(ll), C.c_int]
    L.sp_take_finished.argtypes = [vp, C.POINTER(ll), C.c_int]
    L.sp_failed.argtypes = [vp, ll, d]
    L.sp_advanced.argtypes = [vp, ll]
    L.sp_steps_to_next_check.restype = ll
    L.sp_steps_to_next_check.argtypes = [vp]
    L.sp_checked.restype = C.c_int
    L.sp_checked.argtypes = [vp, ll, d, C.c_int, d, C.c_int, d]
    L.sp_job.restype = C.c_int
    L.sp_job.argtypes = [vp, ll, C.POINTER(C.c_int), C.POINTER(ll), C.POINTER(d), C.POINTER(d)]
    for name in ("sp_running", "sp_queued"):
        getattr(L, name).restype = C.c_int
        getattr(L, name).argtypes = [vp]
    L.sp_bytes.restype = C.c_ulonglong
    L.sp_bytes.argtypes = [vp]
    L.sp_running_nodes.restype = ll
    L.sp_running_nodes.argtypes = [vp]
    return L


class Policy:
    def __init__(self, L, budget, target_nodes=0, max_running=0, check_every=1000, tol_D=1e-4,
                 max_steps=100000):
        self.L = L
        self.h = L.sp_create(budget, target_nodes, max_running, check_every, tol_D, max_steps)

    def __del__(self):
        self.L.sp_destroy(self.h)

    def _ids(self, fn, *a):
        buf = (C.c_longlong * 4096)()
        n = fn(self.h, *a, buf, 4096)
        return [buf[i] for i in range(n)]

    def submit(self, nodes, nbytes, t=0.0):
        return self.L.sp_submit(self.h, nodes, nbytes, t)

    def admit(self, t=0.0):
        return self._ids(self.L.sp_admit, t)

    def due(self):
        return self._ids(self.L.sp_due)

    def finished(self):
        return self._ids(self.L.sp_take_finished)

    def advanced(self, k):
        self.L.sp_advanced(self.h, k)

    def next_check(self):
        return self.L.sp_steps_to_next_check(self.h)

    def checked(self, rid, D, components=1, count=10.0, status=0, t=0.0):
        return self.L.sp_checked(self.h, rid, D, components, count, status, t)

    def failed(self, rid, t=0.0):
        self.L.sp_failed(self.h, rid, t)

    def job(self, rid):
        o, s, ta, td = C.c_int(), C.c_longlong(), C.c_double(), C.c_double()
        assert self.L.sp_job(self.h, rid, C.byref(o), C.byref(s), C.byref(ta), C.byref(td))
        return {"outcome": o.value, "steps": s.value, "t_admit": ta.value, "t_done": td.value}

    def running(self):
        return self.L.sp_running(self.h)

    def queued(self):
        return self.L.sp_queued(self.h)

    def bytes(self):
        return self.L.sp_bytes(self.h)


def test_fifo_admission_under_budget(sp):
    p = Policy(sp, budget=100)
    a, b, c = (p.submit(10, 40) for _ in range(3))
    assert p.admit(1.0) == [a, b]
    assert p.queued() == 1 and p.bytes() == 80
    p.advanced(1000)
    assert sorted(p.due()) == [a, b]
    assert p.checked(a, 0.10, t=2.0) == RUNNING
    p.failed(b, t=2.0)  # the executor lost b
    assert p.bytes() == 40
    assert p.admit(2.5) == [c]
    assert p.job(c)["t_admit"] == 2.5
    assert p.finished() == [b] and p.job(b)["outcome"] == FAILED


def test_oversize_request_is_rejected_at_submit(sp):
    p = Policy(sp, budget=100)
    big = p.submit(10, 101)
    zero = p.submit(10, 0)  # invalid parameters come in with zero bytes
    ok = p.submit(10, 100)
    assert p.finished() == [big, zero]
    assert p.job(big)["outcome"] == REJECTED and p.job(zero)["outcome"] == REJECTED
    assert p.admit() == [ok]


def test_head_of_line_blocks_later_requests(sp):
    """First come first served: a request that does not fit waits and the
    ones behind it wait too."""
    p = Policy(sp, budget=100)
    a = p.submit(10, 60)
    b = p.submit(10, 60)
    c = p.submit(10, 10)
    assert p.admit() == [a]
    assert p.admit() == []
    p.failed(a)
    assert p.admit() == [b, c]


def test_running_limits(sp):
    p = Policy(sp, budget=10**6, max_running=1)
    ids = [p.submit(5, 10) for _ in range(3)]
    assert p.admit() == ids[:1]
    assert p.admit() == []
    q = Policy(sp, budget=10**6, target_nodes=25)
    ids = [q.submit(10, 10) for _ in range(4)]
    assert q.admit() == ids[:2]  # a third would make 30 > 25 nodes
    r = Policy(sp, budget=10**6, target_nodes=5)
    big = r.submit(50, 10)
    assert r.admit() == [big]  # an idle server always starts the head request


def test_convergence_rule(sp):
    """Converged at the first check whose |D - D_prev| < tol_D, never at the
    first check; checks every check_every steps of the request."""
    p = Policy(sp, budget=100, check_every=1000, tol_D=1e-4)
    a = p.submit(10, 10)
    p.admit()
    trajectory = [0.05, 0.08, 0.0900, 0.09005]
    outs = []
    for D in trajectory:
        assert p.next_check() == 1000
        p.advanced(600)
        assert p.due() == []
        assert p.next_check() == 400
        p.advanced(400)
        assert p.due() == [a]
        outs.append(p.checked(a, D))
    assert outs == [RUNNING, RUNNING, RUNNING, CONVERGED]
    assert p.job(a)["steps"] == 4000 and p.running() == 0 and p.bytes() == 0
    # a constant D converges at the second check, not the first
    b = p.submit(10, 10)
    p.admit()
    p.advanced(1000)
    assert p.checked(b, 0.2) == RUNNING
    p.advanced(1000)
    assert p.checked(b, 0.2) == CONVERGED


def test_breakup_unstable_and_cap(sp):
    p = Policy(sp, budget=1000, check_every=100, max_steps=250)
    a = p.submit(1, 10)
    b = p.submit(1, 10)
    c = p.submit(1, 10)
    d = p.submit(1, 10)
    p.admit()
    p.advanced(100)
    assert p.checked(a, 0.3, components=2) == BREAKUP  # the drop split in two
    assert p.checked(b, 0.3, count=0.0) == BREAKUP  # no liquid left
    assert p.checked(c, 0.3, status=1) == UNSTABLE
    assert p.checked(d, 0.3) == RUNNING
    p.advanced(100)
    assert p.checked(d, 0.1) == RUNNING
    assert p.next_check() == 50  # the cap comes before the next check
    p.advanced(50)
    assert p.due() == [d]
    assert p.checked(d, 0.3) == MAX_STEPS
    assert [p.job(x)["outcome"] for x in (a, b, c, d)] == [BREAKUP, BREAKUP, UNSTABLE, MAX_STEPS]
    assert p.finished() == [a, b, c, d]


def test_fake_executor_with_injected_failures(sp):
    """A whole serving run with a fake executor: random arrivals and sizes,
    scripted deformation histories, and failures injected on the host (every
    7th start fails, every 11th request is lost after its first check).
    Invariants: the budget is never exceeded, every request finishes exactly
    once, admission follows arrival order, and everything is released."""
    rng = np.random.default_rng(7)
    budget = 1000
    p = Policy(sp, budget=budget, check_every=100, tol_D=1e-3, max_steps=5000)
    n_req = 120
    arrivals = np.cumsum(rng.exponential(1.0, n_req))
    sizes = rng.integers(50, 400, n_req)
    conv_at = rng.integers(2, 12, n_req)  # checks until D settles
    ids, admitted, finished = [], [], []
    checks = {}
    starts = 0
    t, i = 0.0, 0
    while len(finished) < n_req:
        while i < n_req and arrivals[i] <= t:
            ids.append(p.submit(int(sizes[i]), int(sizes[i]), t))
            i += 1
        for rid in p.admit(t):
            starts += 1
            admitted.append(rid)
            if starts % 7 == 0:
                p.failed(rid, t)  # executor could not start it
        assert p.bytes() <= budget
        if p.running():
            k = min(40, p.next_check())
            p.advanced(k)
            for rid in p.due():
                n = checks.get(rid, 0) + 1
                checks[rid] = n
                if rid % 11 == 0 and n == 1:
                    p.failed(rid, t)  # lost while running
                    continue
                k_req = ids.index(rid)
                D = 0.3 if n >= conv_at[k_req] else 0.3 - 0.01 * (conv_at[k_req] - n)
                p.checked(rid, D, t=t)
        finished += p.finished()
        t += 0.5
    assert sorted(finished) == sorted(ids) and len(set(finished)) == n_req
    assert admitted == sorted(admitted)  # FIFO
    assert p.bytes() == 0 and p.running() == 0 and p.queued() == 0
    outcomes = [p.job(r)["outcome"] for r in ids]
    assert outcomes.count(FAILED) >= n_req // 11
    assert all(o in (CONVERGED, FAILED) for o in outcomes)
    for r in ids:
        j = p.job(r)
        if j["outcome"] == CONVERGED:
            k_req = ids.index(r)
            # D settles at check conv_at; the next check sees |dD| = 0
            assert j["steps"] == 100 * (int(conv_at[k_req]) + 1)
