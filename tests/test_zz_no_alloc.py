"""The allocation-free adjoint sweep against the allocating one.

stc_adjoint_sweep_noalloc serves callers that cannot allocate device memory
when they run the sweep (a process whose device memory is reserved up front
by its own pool, or a caller that cannot afford cudaMalloc's implicit
synchronisation); it keeps its scratch in a fixed device array.  Here its
output, through the C ABI, must equal that of stc_adjoint of a problem on the
same inputs, on two calls in a row (the second sees the first's leftovers in
the shared scratch).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1608_01102_gb300 import stc, workloads

from gpu_common import TOL, make_pair, rel, velocity_trajectory

pytestmark = pytest.mark.gpu


def test_noalloc_sweep_matches_problem_sweep_twice():
    torch = pytest.importorskip("torch")
    nx, ny, N = 32, 24, 6
    kf = {N // 2: (workloads.gaussian_ball(nx, ny, (0.4, 0.4), 0.1), 0.5),
          N: (workloads.gaussian_ball(nx, ny, (0.6, 0.5), 0.1), 1.0)}
    P, G = make_pair(nx, ny, N=N, precision=0, levels=2, keyframes=kf, K=2.0)
    v = velocity_trajectory(nx, ny, N, amp=0.7, seed=3)
    w = workloads.random_faces(np.random.default_rng(4), nx, ny, N, 0.2)
    G.set("VSTAR", v[:N])
    G.set("W", w)
    G.advect("VSTAR")
    G.metric_terms()
    G.adjoint("VSTAR", 1.0, 1.0 / P.K)          # the allocating path
    mu_ref, y_ref = G.get("MU"), G.get("Y")

    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    vel = torch.tensor(G.get("VSTAR"), **f32)
    rho = torch.tensor(G.get("RHO"), **f32)
    Ks = torch.tensor(G.taylor_orders(), dtype=torch.int32, device=dev)
    mterm = torch.tensor(G.get("MTERM"), dtype=torch.float64, device=dev)
    base = torch.tensor(G.get("W"), **f32)
    stream = torch.cuda.current_stream()
    for call in range(2):
        mu = torch.full((N, nx * ny), float("nan"), **f32)
        out = torch.full_like(vel, float("nan"))
        stc.adjoint_sweep_noalloc(nx, ny, N, P.dt, G.taylor_kmax(), vel.data_ptr(), rho.data_ptr(),
                                  Ks.data_ptr(), mterm.data_ptr(), mu.data_ptr(), base.data_ptr(), 1.0,
                                  1.0 / P.K, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        mu_h, out_h = mu.cpu().numpy(), out.cpu().numpy()
        for s in range(N):
            assert rel(mu_h[s], mu_ref[s]) < TOL[0]["exact"], (call, s)
        for s in range(1, N):
            assert rel(out_h[s], y_ref[s]) < TOL[0]["exact"], (call, s)


def test_noalloc_rejects_scratch_beyond_the_fixed_size():
    torch = pytest.importorskip("torch")
    t = torch.zeros(16, device="cuda")
    p = t.data_ptr()
    with pytest.raises(stc.StcError) as e:
        stc.adjoint_sweep_noalloc(128, 128, 4, 0.25, 65, p, p, p, p, p, None, 1.0, 1.0, p)
    assert "1048576" in str(e.value)


def test_noalloc_reports_an_order_above_taylor_kmax():
    """Orders from a forward sweep run with a larger taylor_kmax than the one
    passed are reported (STC_ERR_DIVERGED), not silently truncated; the next
    call with valid orders succeeds (each call clears the error word)."""
    torch = pytest.importorskip("torch")
    nx, ny, N, kmax = 16, 16, 3, 8
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    F = workloads.face_count(nx, ny)
    vel = torch.zeros((N, F), **f32)
    rho = torch.ones((N + 1, nx * ny), **f32)
    mterm = torch.zeros((N + 1, nx * ny), dtype=torch.float64, device=dev)
    mu = torch.zeros((N, nx * ny), **f32)
    out = torch.zeros((N, F), **f32)
    stream = torch.cuda.current_stream().cuda_stream
    bad = torch.tensor([1, kmax + 1, 1], dtype=torch.int32, device=dev)
    with pytest.raises(stc.StcError) as e:
        stc.adjoint_sweep_noalloc(nx, ny, N, 1.0 / N, kmax, vel.data_ptr(), rho.data_ptr(), bad.data_ptr(),
                                  mterm.data_ptr(), mu.data_ptr(), None, 0.0, 1.0, out.data_ptr(), stream)
    assert e.value.code == 5 and "taylor_kmax" in str(e.value)
    good = torch.tensor([1, kmax, 1], dtype=torch.int32, device=dev)
    stc.adjoint_sweep_noalloc(nx, ny, N, 1.0 / N, kmax, vel.data_ptr(), rho.data_ptr(), good.data_ptr(),
                              mterm.data_ptr(), mu.data_ptr(), None, 0.0, 1.0, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.all(mu == 0) and torch.all(out[1:] == 0)
