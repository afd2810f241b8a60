"""Serving on the GPU (include/stc_server.h): problems of different grid sizes,
timestep counts and keyframe sets solved concurrently give the same result as
each solved alone; the admission size equals the bytes a problem holds."""
import numpy as np
import pytest

from paper_1608_01102_gb300 import stc, workloads

pytestmark = pytest.mark.gpu

CASES = [(16, 16, 6, 1), (32, 32, 8, 2), (16, 16, 10, 2), (24, 24, 6, 1)]


def _problem(nx, ny, N, nkeys, prec):
    prm = stc.default_params(nx, ny, N, precision=prec, r=1e-2, metric_levels=2)
    rho0 = workloads.gaussian_ball(nx, ny, (0.5, 0.3), 0.12)
    kf = {}
    for j in range(1, nkeys + 1):
        step = round(j * N / nkeys)
        kf[step] = (workloads.gaussian_ball(nx, ny, (0.5, 0.3 + 0.35 * j / nkeys), 0.12), 1.0)
    return prm, rho0, kf


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", [1, 0])
def test_each_result_is_the_same_alone_and_in_the_mix(prec):
    alone = []
    for (nx, ny, N, nk) in CASES:
        prm, rho0, kf = _problem(nx, ny, N, nk, prec)
        with stc.Problem(prm, rho0) as G:
            G.set_keyframes(kf)
            rep = G.solve(tol=1e-6, max_admm=6)
            alone.append((rep, G.forces()))
    budget = sum(stc.problem_bytes(_problem(*c, prec)[0], c[3]) for c in CASES)
    with stc.Server(budget, workers=len(CASES)) as S:
        tickets = [S.submit(*_problem(*c, prec), tol=1e-6, max_admm=6) for c in CASES]
        infos = [S.wait(t) for t in tickets]
        assert S.stats()["peak_bytes"] <= budget
        seen = [(i["report"]["admm_iters"], i["report"]["vcycles"]) for i in infos]
        ref = [(r["admm_iters"], r["vcycles"]) for r, _ in alone]
        for t, info, (rep, u) in zip(tickets, infos, alone):
            assert info["state"] == "done", info
            assert info["report"]["admm_iters"] == rep["admm_iters"], (seen, ref)
            assert info["report"]["vcycles"] == rep["vcycles"], (seen, ref)
            got = S.forces(t)
            assert _rel(got, u) <= (1e-9 if prec == 1 else 1e-5), _rel(got, u)
            assert abs(info["report"]["kkt_rel"] - rep["kkt_rel"]) <= 1e-6 * rep["kkt_rel"] + 1e-12


@pytest.mark.parametrize("prec", [1, 0])
def test_admission_size_is_the_memory_a_problem_holds(prec):
    # (fp64 state at 128^2 exceeds the on-chip projection's shared memory: fp32 only)
    big = [(128, 128, 40, 1)] if prec == 0 else []
    for (nx, ny, N, nk) in CASES + big + [(64, 64, 48, 3)]:
        prm, rho0, kf = _problem(nx, ny, N, nk, prec)
        with stc.Problem(prm, rho0) as G:
            G.set_keyframes(kf)
            assert G.memory_bytes() == stc.problem_bytes(prm, nk), (nx, N, nk)


@pytest.mark.parametrize("prec", [1, 0])
def test_batched_steps_give_each_result_as_alone(prec):
    """Stepped serving (mode 1): every step runs the next NSO V-cycle of all
    resident problems in one batched graph launch, and problems are admitted
    and retired between steps.  Each result equals the problem solved alone
    (same iterations, V-cycles, residual and forces), with a budget that
    holds only some of the problems at once (continuous admission) and with a
    caller-created problem submitted beside the requests."""
    torch = pytest.importorskip("torch")
    alone = []
    for (nx, ny, N, nk) in CASES:
        prm, rho0, kf = _problem(nx, ny, N, nk, prec)
        with stc.Problem(prm, rho0) as G:
            G.set_keyframes(kf)
            rep = G.solve(tol=1e-6, max_admm=6)
            alone.append((rep, G.forces()))
    sizes = [stc.problem_bytes(_problem(*c, prec)[0], c[3]) for c in CASES]
    budget = sum(sorted(sizes)[-2:])        # at most about two problems at once
    stream = torch.cuda.Stream()
    with stc.Server(budget, mode=1, stream=stream.cuda_stream, max_resident=3, tol=1e-6, max_admm=6) as S:
        tickets = [S.submit(*_problem(*c, prec), tol=1e-6, max_admm=6) for c in CASES[:-1]]
        prm, rho0, kf = _problem(*CASES[-1], prec)
        own = stc.Problem(prm, rho0, stream=stream.cuda_stream)
        own.set_keyframes(kf)
        tickets.append(S.submit_problem(own))
        steps, max_running = 0, 0
        while S.step() > 0:
            steps += 1
            max_running = max(max_running, S.stats()["running"])
            assert steps < 2000
        assert 1 < max_running <= 3 and S.stats()["peak_bytes"] <= budget
        for t, (rep, u) in zip(tickets, alone):
            info = S.poll(t)
            assert info["state"] == "done", info
            assert info["report"]["admm_iters"] == rep["admm_iters"]
            assert info["report"]["vcycles"] == rep["vcycles"]
            assert _rel(S.forces(t), u) <= (1e-9 if prec == 1 else 1e-5)
            assert abs(info["report"]["kkt_rel"] - rep["kkt_rel"]) <= 1e-6 * rep["kkt_rel"] + 1e-12
        assert _rel(own.forces(), alone[-1][1]) <= (1e-9 if prec == 1 else 1e-5)
        own.close()
