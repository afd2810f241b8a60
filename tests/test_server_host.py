"""Serving scheduler (include/stc_server.h) on the simulated backend: admission
against the memory budget, first fit with a bypass limit, cancellation,
failure isolation and shutdown -- host logic only, no CUDA call, no GPU.
The admission size stc_problem_bytes is checked here against the memory
bound of Sec. 5 and, on a GPU, against the bytes a problem really holds."""
import time

import numpy as np
import pytest

from paper_1608_01102_gb300 import build, stc, workloads


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    stc.load()


def _req(n, N):
    prm = stc.default_params(n, n, N)
    rho0 = workloads.gaussian_ball(n, n, (0.5, 0.3), 0.08)
    return prm, rho0, {N: (rho0, 1.0)}


def test_problem_bytes_scale_like_the_papers_memory_bound():
    """Sec. 5: STFAS memory M ~ 8 n^d (1 + d) N scalars.  The admission size
    grows linearly in N and in n^d, doubles (to within the fixed int/fp64
    buffers) from fp32 to fp64 storage, and stays within a fixed multiple of M."""
    b = {}
    for n in (32, 64, 128):
        for N in (16, 32):
            prm = stc.default_params(n, n, N)
            b[n, N] = stc.problem_bytes(prm, 1)
            M = 8 * n * n * 3 * N
            assert 1.0 <= b[n, N] / (4 * M) <= 4.0, (n, N, b[n, N] / (4 * M))
    assert 1.8 < b[64, 32] / b[64, 16] < 2.1
    assert 3.6 < b[128, 16] / b[64, 16] < 4.2
    prm64 = stc.default_params(64, 64, 16, precision=1)
    assert 1.7 < stc.problem_bytes(prm64, 1) / b[64, 16] < 2.1
    assert stc.problem_bytes(stc.default_params(64, 64, 16), 3) - b[64, 16] == 2 * 64 * 64 * 8
    with pytest.raises(stc.StcError):
        stc.problem_bytes(stc.default_params(64, 64, 0), 1)


def test_admission_never_exceeds_the_budget_and_everything_completes():
    sizes = [(32, 16), (64, 24), (48, 16), (64, 32), (32, 48), (64, 16)]
    need = [stc.problem_bytes(_req(n, N)[0], 1) for n, N in sizes]
    budget = max(need) + min(need)          # at most ~2 resident at a time
    with stc.Server(budget, workers=4, backend=1) as S:
        tickets = []
        for (n, N) in sizes:
            prm, rho0, kf = _req(n, N)
            tickets.append(S.submit(prm, rho0, kf, sim_seconds=0.05))
        peak_running = 0
        while True:
            st = S.stats()
            peak_running = max(peak_running, st["running"])
            assert st["bytes_in_use"] <= budget
            if st["done"] == len(sizes):
                break
            time.sleep(0.005)
        assert S.stats()["peak_bytes"] <= budget
        assert peak_running >= 2             # problems did overlap
        for t, (n, N) in zip(tickets, sizes):
            info = S.wait(t)
            assert info["state"] == "done" and info["t_submit"] <= info["t_admit"] <= info["t_done"]
            assert S.forces(t).shape == (N, n * (n + 1) * 2)
            S.release(t)


def test_first_fit_passes_a_big_request_but_only_max_bypass_times():
    small = _req(32, 16)
    big = _req(64, 32)
    sb = stc.problem_bytes(small[0], 1)
    bb = stc.problem_bytes(big[0], 1)
    budget = bb + sb // 2                     # big fits only when nothing else runs
    with stc.Server(budget, workers=4, backend=1, max_bypass=2) as S:
        first = S.submit(*small, sim_seconds=0.3)       # occupies part of the budget
        time.sleep(0.05)
        tb = S.submit(*big, sim_seconds=0.01)            # does not fit yet
        ts = [S.submit(*small, sim_seconds=0.01) for _ in range(4)]
        infos = [S.wait(t) for t in ts]
        ib = S.wait(tb)
        S.wait(first)
        admits = sorted(i["t_admit"] for i in infos)
        # two small requests overtake the big one, the rest wait behind it
        assert sum(a < ib["t_admit"] for a in admits) == 2, (admits, ib["t_admit"])
        assert all(i["state"] == "done" for i in infos + [ib])


def test_oversize_malformed_failed_and_cancelled_requests():
    prm, rho0, kf = _req(32, 16)
    need = stc.problem_bytes(prm, 1)
    with stc.Server(need, workers=1, backend=1) as S:
        with pytest.raises(stc.StcError) as e:
            S.submit(*_req(64, 16))
        assert e.value.code == 2                         # never admissible: OOM at submit
        with pytest.raises(stc.StcError) as e:
            S.submit(prm, rho0, {0: kf[16]})             # keyframe step outside 1..N
        assert e.value.code == 1
        bad = S.submit(prm, rho0, kf, sim_seconds=0.05, sim_status=3)   # a failing solve
        a = S.submit(prm, rho0, kf, sim_seconds=0.05)
        b = S.submit(prm, rho0, kf, sim_seconds=0.05)
        S.cancel(b)
        ib = S.wait(bad)
        assert ib["state"] == "failed" and ib["status"] == 3 and ib["error"]
        with pytest.raises(stc.StcError):
            S.forces(bad)
        assert S.wait(a)["state"] == "done"              # the failure did not spread
        assert S.wait(b)["state"] == "cancelled"
        c = S.submit(prm, rho0, kf, sim_seconds=0.3)
        while S.poll(c)["state"] != "running":
            time.sleep(0.005)
        with pytest.raises(stc.StcError) as e:
            S.cancel(c)
        assert e.value.code == 7                         # running requests are not interrupted
        st = S.stats()
        assert st["failed"] == 1 and st["cancelled"] == 1


def test_shutdown_cancels_the_queue_and_waits_for_running_solves():
    prm, rho0, kf = _req(32, 16)
    S = stc.Server(stc.problem_bytes(prm, 1), workers=1, backend=1)
    t1 = S.submit(prm, rho0, kf, sim_seconds=0.2)
    [S.submit(prm, rho0, kf, sim_seconds=0.2) for _ in range(3)]
    while S.poll(t1)["state"] != "running":
        time.sleep(0.005)
    t0 = time.perf_counter()
    S.close()
    assert time.perf_counter() - t0 < 1.0                # only the running one was waited for
