"""The forward smoke simulation as a differentiable PyTorch function.

``simulate(u, sim)`` maps the control forces u (N x faces, a CUDA tensor) to
the densities rho_0..rho_N ((N+1) x cells): every step solves the implicit
Navier-Stokes step of Eq. NSA/NSB under u_i (stc_simulate: Picard iteration
with the library's projection) and advects the density with the Taylor
exponential (Eq. Conv).  Its backward pass is the library's hand-written
adjoint (stc_simulate_adjoint: the backward density sweep of Eq. KKTPO and
the transposed implicit step), so ``loss.backward()`` yields dL/du.

With ``checkpoint_every = k`` the trajectory is cut into segments of k steps:
the forward pass keeps only each segment's starting velocity and density, and
the backward pass recomputes one segment at a time (a problem of k steps)
before running its adjoint, chaining the adjoints of v and rho across the
segment boundaries.  Device memory then scales with k instead of N.

PyTorch supplies device memory and the stream; every step runs in libstc's
kernels (no CPU fallback: stc.load() raises if the library is missing).
"""
import torch

from . import stc


class Simulation:
    """Geometry and numerics of the differentiable simulation (one GPU).

    nx, ny, nz (0 for 2D), N steps of dt; rho0 (cells) and v0 (faces or None)
    as numpy arrays; precision 0 (fp32) or 1 (fp64); picard_tol relative."""

    def __init__(self, nx, ny, N, rho0, v0=None, nz=0, dt=None, precision=0, picard_tol=None, max_iter=200,
                 taylor_tol=1e-5, checkpoint_every=None):
        self.nx, self.ny, self.nz, self.N = nx, ny, nz, N
        self.dt = 1.0 / N if dt is None else dt
        self.precision = precision
        self.dtype = torch.float64 if precision == 1 else torch.float32
        self.picard_tol = picard_tol if picard_tol is not None else (1e-12 if precision == 1 else 1e-6)
        self.max_iter = max_iter
        self.taylor_tol = taylor_tol
        self.F, self.C = stc.grid_sizes(nx, ny, nz)
        self.rho0 = torch.as_tensor(rho0, dtype=self.dtype).reshape(self.C)
        self.v0 = (torch.zeros(self.F, dtype=self.dtype) if v0 is None
                   else torch.as_tensor(v0, dtype=self.dtype).reshape(self.F))
        self.rho_scale = float(self.rho0.abs().max())
        k = checkpoint_every or N
        self.segments = [(s, min(s + k, N)) for s in range(0, N, k)]
        self._problems = {}
        self.picard_iterations = 0

    def problem(self, steps):
        """A library problem of `steps` steps (kept for reuse)."""
        if steps not in self._problems:
            prm = stc.default_params(self.nx, self.ny, steps, precision=self.precision, dt=self.dt, nz=self.nz,
                                     taylor_tol=self.taylor_tol)
            # Taylor truncation relative to the full problem's initial density
            # (the same threshold in every segment)
            rho0 = self.rho0.detach().cpu().double().numpy()
            self._problems[steps] = stc.Problem(prm, rho0, stream=torch.cuda.current_stream().cuda_stream)
        return self._problems[steps]

    def close(self):
        for p in self._problems.values():
            p.close()
        self._problems = {}


def _put(G, name, t, scale=1.0):
    t = t.contiguous()
    G.copy_device(name, t.data_ptr(), t.numel(), t.dtype == torch.float64, True, scale)


def _get(G, name, t, scale=1.0):
    G.copy_device(name, t.data_ptr(), t.numel(), t.dtype == torch.float64, False, scale)


def _run_segment(sim, G, v_start, rho_start, u_seg):
    """Simulate one segment on problem G from (v_start, rho_start) under u_seg;
    returns (rho (k+1) x C, v_end)."""
    k = u_seg.shape[0]
    dev = u_seg.device
    v = torch.zeros((k + 1, sim.F), dtype=sim.dtype, device=dev)
    v[0] = v_start
    rho = torch.zeros((k + 1, sim.C), dtype=sim.dtype, device=dev)
    rho[0] = rho_start
    _put(G, "V", v)
    _put(G, "RHO", rho)
    _put(G, "U", u_seg)
    sim.picard_iterations += G.simulate(sim.picard_tol, sim.max_iter)
    _get(G, "RHO", rho)
    _get(G, "V", v)
    return rho, v[k].clone()


class _SimulateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, sim):
        u = u.detach().to(sim.dtype).contiguous()
        dev = u.device
        v = sim.v0.to(dev)
        rho0 = sim.rho0.to(dev)
        starts = []           # (v, rho) at every segment start: the checkpoints
        out = torch.empty((sim.N + 1, sim.C), dtype=sim.dtype, device=dev)
        out[0] = rho0
        r = rho0
        for (a, b) in sim.segments:
            starts.append((v.clone(), r.clone()))
            G = sim.problem(b - a)
            rho_seg, v = _run_segment(sim, G, v, r, u[a:b])
            out[a + 1:b + 1] = rho_seg[1:]
            r = rho_seg[-1]
        ctx.sim = sim
        ctx.save_for_backward(u, *[t for pair in starts for t in pair])
        return out

    @staticmethod
    def backward(ctx, grad_rho):
        sim = ctx.sim
        saved = ctx.saved_tensors
        u = saved[0]
        starts = [(saved[1 + 2 * i], saved[2 + 2 * i]) for i in range(len(sim.segments))]
        dev = u.device
        grad_rho = grad_rho.to(torch.float64).contiguous()
        grad_u = torch.zeros_like(u)
        a_v = torch.zeros(sim.F, dtype=sim.dtype, device=dev)       # dL/dv at the segment end
        l_rho = torch.zeros(sim.C, dtype=torch.float64, device=dev)  # dL/drho at the segment end (from later)
        for idx in range(len(sim.segments) - 1, -1, -1):
            a, b = sim.segments[idx]
            G = sim.problem(b - a)
            v_start, r_start = starts[idx]
            _run_segment(sim, G, v_start, r_start, u[a:b])          # recompute this segment
            g = grad_rho[a:b + 1].clone()
            g[-1] += l_rho                                          # adjoint carried from the next segment
            if idx > 0:
                g[0] = 0.0     # rho_a's direct term belongs to the previous segment's end
            _put(G, "SIM_GRAD_RHO", g)
            _put(G, "SIM_ADJ_VN", a_v)
            sim.picard_iterations += G.simulate_adjoint(sim.picard_tol, sim.max_iter, with_step0=idx > 0)
            gu = torch.empty((b - a, sim.F), dtype=sim.dtype, device=dev)
            _get(G, "SIM_GRAD_U", gu)
            grad_u[a:b] = gu
            a0 = torch.empty(sim.F, dtype=sim.dtype, device=dev)
            _get(G, "SIM_ADJ_V0", a0)
            a_v = a0
            if idx > 0:
                l0 = torch.empty(sim.C, dtype=torch.float64, device=dev)
                _get(G, "SIM_ADJ_RHO0", l0)
                l_rho = l0
        return grad_u, None


def simulate(u, sim):
    """rho_0..rho_N ((N+1) x cells) of the simulation driven by u (N x faces)."""
    return _SimulateFn.apply(u, sim)
