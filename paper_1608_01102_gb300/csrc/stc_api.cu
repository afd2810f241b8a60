// Host orchestration and C ABI of libstc (see include/stc.h).
//
// The STFAS V-cycle (Alg. 2) is enqueued as a fixed sequence of kernels and
// captured once into a CUDA graph, then replayed; the AO fixed point (Alg. 1),
// the KKT metric and the ADMM loop (Alg. 3) are enqueued on the problem's
// stream.  Host code only marshals arguments, sequences launches and reads
// back fp64 scalars for the stopping tests.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <limits>
#include <vector>

#include "../../include/stc.h"
#include "stc_internal.cuh"
#include "stc_kernels.h"

using namespace stc;

namespace {

thread_local std::string g_last_error;

struct FieldSet {
  void* v = nullptr;
  void* pbar = nullptr;
  void* u = nullptr;
  void* p = nullptr;
};

struct Level {
  Geom g;
  bool dbl = false;
  FieldSet x, res, tmp, old;
  void* z = nullptr;
};

template <class T>
State<T> st_of(const FieldSet& f) {
  return State<T>{(T*)f.v, (T*)f.pbar, (T*)f.u, (T*)f.p};
}
template <class T>
CState<T> cst_of(const FieldSet& f) {
  return CState<T>{(const T*)f.v, (const T*)f.pbar, (const T*)f.u, (const T*)f.p};
}

template <class F>
void dispatch(bool dbl, F&& f) {
  if (dbl) f(double());
  else f(float());
}

struct StcError {
  stc_status code;
  std::string msg;
};

[[noreturn]] void fail(stc_status code, const std::string& msg) { throw StcError{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(STC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

void stc::set_last_error(const char* msg) { g_last_error = msg; }

constexpr int kMaxTrials = 8;   // most AO blend factors tried at once

// The ADMM loop of one stc_solve (Alg. 3) as resumable phases, so that a
// serving step can run the V-cycles of many problems in one graph launch.
struct SolveRun {
  int phase = 2;                  // 0: an iteration begins (AO due); 1: NSO V-cycles due; 2: finished
  double tol = 1e-4;
  int max_admm = 0;
  std::chrono::steady_clock::time_point t0;
  double K0 = 0.0, g0 = 0.0, J_prev = 0.0, eps_admm = 0.0, f = 0.0;
  bool have_prev = false;         // k_adapt: v_prev holds a previous iteration's v
  bool give_up = false;           // the NSO solve ends (a cycle undone at the largest LM shift)
  bool converged = false;
  int it = 0, cycles = 0;
  stc_report rep{};
};

struct stc_problem {
  stc_params prm;
  cudaStream_t st = nullptr;      // user stream (may be the legacy default)
  cudaStream_t cap = nullptr;     // private stream used only to capture graphs
  bool dbl = false;               // finest-level type is double
  size_t ts = 4;
  std::vector<Level> lv;
  std::vector<void*> allocs;
  void *rho = nullptr, *rho_k = nullptr, *rho_last = nullptr, *mu = nullptr, *vstar = nullptr, *lam = nullptr,
       *w = nullptr, *y = nullptr, *uk = nullptr, *gk = nullptr, *dens = nullptr, *powers = nullptr,
       *v0 = nullptr;
  void *vcand = nullptr, *rho_c = nullptr;   // AO blend trial: v*, its densities and Taylor orders
  void* vprev = nullptr;          // k_adapt: v of the previous ADMM iteration
  int *K = nullptr, *Kk = nullptr, *K_c = nullptr;
  // concurrent AO blend trials (2D): trial j's v*, densities, orders, metric
  // terms, metric temporaries, error flags and objective; trial 0 is
  // vcand / rho_c / K_c (and mtmp0 / mtmp1)
  int ntrials = 1;
  void* tv[kMaxTrials] = {};
  void* trho[kMaxTrials] = {};
  int* tK[kMaxTrials] = {};
  double* tmterm[kMaxTrials] = {};
  double* ttmp0[kMaxTrials] = {};
  double* ttmp1[kMaxTrials] = {};
  int* terr = nullptr;
  double* dtrial = nullptr;
  void* htrial = nullptr;         // pinned: kMaxTrials doubles, then kMaxTrials ints
  cudaStream_t tst[kMaxTrials] = {};
  cudaStream_t aux = nullptr;     // second stream of the KKT evaluation (force branch)
  cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
  cudaEvent_t tfork = nullptr;
  cudaEvent_t tdone[kMaxTrials] = {};
  bool rho_at_vstar = false;      // rho / K hold the forward sweep of the current v*
  std::vector<int> ao_trace;      // halvings per pass of the last AO
  std::vector<double> solve_hist; // last stc_solve: per ADMM iteration (kkt_rel, seconds, K)
  SolveRun run;                   // the solve in progress (or the last one)
  cudaGraph_t vgraph_src = nullptr;   // the captured plain V-cycle (child node of batched launches)
  long long vgraph_version = 0;   // bumped at every capture of vgraph
  double* dguard = nullptr;       // per level {before, after} ||res - f||_2^2 of the guarded correction
  double* dlm = nullptr;          // device copy of the smoother's LM shift gamma (read by every SCGS launch)
  double lm0 = 0.0, lm = 0.0;     // default and current gamma
  FieldSet xb;                    // finest state before the last V-cycle (undo of a rejected cycle)
  int rejected = 0;               // V-cycles undone by the LM safeguard
  double *mterm = nullptr, *mtmp0 = nullptr, *mtmp1 = nullptr, *star = nullptr;
  size_t star_bytes = 0;
  void* pscratch = nullptr;       // projection level arrays when they do not fit on chip
  void* dct = nullptr;            // 2D: DCT tables of the exact projection (project_dct_tables, state type)
  void* adv3 = nullptr;           // 3D sweeps: term buffers and grid-barrier words
  void* sc3 = nullptr;            // 3D SCGS: per-cell block Thomas records (finest level's size)
  void* lamb3 = nullptr;          // 3D: two-pass residual scratch (finest level's size; large levels only)
  size_t lamb3_bytes = 0;
  // forward simulation and its adjoint (allocated at their first use)
  void *sim_gu = nullptr, *sim_a0 = nullptr, *sim_l0 = nullptr, *sim_aN = nullptr, *sim_w1 = nullptr,
       *sim_w2 = nullptr, *sim_w3 = nullptr;
  double* sim_grho = nullptr;     // dL/d rho_i, i = 0..N (fp64)
  std::vector<int> key_steps;
  std::vector<double> key_c;
  double* dscal = nullptr;  // device fp64 scalars
  double* hscal = nullptr;  // pinned host mirror
  int* derr = nullptr;
  int* herr = nullptr;
  RedScratch red{};               // deterministic sums on the problem's stream
  RedScratch tred[kMaxTrials] = {};   // ... on the blend trials' streams
  double rho_scale = 0.0;
  double fscale = -1.0;
  cudaGraphExec_t vgraph = nullptr;
  cudaGraphExec_t vgraph_t = nullptr;   // the same V-cycle with events around the finest SCGS launches
  bool capture_timed = false;           // capturing vgraph_t
  bool broken = false;
  // instrumentation
  long long launches = 0;       // kernels enqueued (graph replays add graph_launches)
  long long graph_launches = 0; // kernel nodes of the V-cycle graph
  long long* counter = nullptr; // where enqueue sites count: &launches, or &graph_launches while capturing
  bool timing = false;
  // kind 0: the finest level's SCGS colour launches, kind 1: its colour residuals
  std::vector<cudaEvent_t> ev_start[2], ev_stop[2];
  int ev_used[2] = {};          // event pairs recorded by the current graph
  double timed_ms[2] = {};
  long long timed_launches[2] = {};
  size_t bytes = 0;
};

namespace {

void count(stc_problem* P, long long k) { *(P->counter ? P->counter : &P->launches) += k; }

void* dalloc(stc_problem* P, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  P->bytes += bytes;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? STC_ERR_OOM : STC_ERR_CUDA,
         std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  P->allocs.push_back(p);
  ck(cudaMemsetAsync(p, 0, bytes, P->st), "memset");
  return p;
}

// scratch of the deterministic sums: partials for cap blocks and a ticket
RedScratch alloc_red(stc_problem* P, size_t cap) {
  RedScratch r;
  r.part = (double*)dalloc(P, cap * sizeof(double));
  r.ticket = (unsigned*)dalloc(P, sizeof(unsigned));
  r.cap = (unsigned)cap;
  return r;
}

// the most blocks of a reduction on the problem's stream: the finest level's
// residual with its fused norm, or the generic sums
size_t red_capacity(const Geom& g0) {
  const size_t b = nso_residual_blocks(g0);
  return b > kReduceMaxBlocks ? b : kReduceMaxBlocks;
}

// (N, dt: the level's; the smoother's LM shift stays the finest level's;
// nz = 0: the 2D grid, else the 3D grid with nz cells along z)
Geom make_geom(const stc_params& prm, int nx, int ny, int nz, double h, int N, double dt) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.N = N;
  if (nz > 0) {
    g.dim = 3;
    g.nz = nz;
    g.Fx = nz * ny * (nx + 1);
    g.Fy = nz * (ny + 1) * nx;
    g.Fxy = g.Fx + g.Fy;
    g.F = g.Fxy + (nz + 1) * ny * nx;
    g.C = nx * ny * nz;
  } else {
    g.dim = 2;
    g.nz = 1;
    g.Fx = ny * (nx + 1);
    g.Fy = (ny + 1) * nx;
    g.F = g.Fx + g.Fy;
    g.Fxy = g.F;
    g.C = nx * ny;
  }
  g.periodic = (nz > 0 && prm.boundary == 1) ? 1 : 0;
  g.h = h;
  g.ih = 1.0 / h;
  g.dt = dt;
  g.idt = 1.0 / dt;
  g.a = prm.K / prm.r;
  g.lm = prm.lm_shift < 0 ? 1.0 / (prm.dt * prm.dt) : prm.lm_shift;
  g.omega = prm.scgs_omega;
  g.self_adv = prm.self_advection ? 1 : 0;
  g.cta_cells = prm.scgs_cta_cells;
  set_fp32_copies(g);
  return g;
}

// the STFAS hierarchy coarsens while every axis is even and its half stays >= coarsest_n
bool can_halve(const stc_params& prm, int nx, int ny, int nz) {
  const bool xy = nx % 2 == 0 && ny % 2 == 0 && nx / 2 >= prm.coarsest_n && ny / 2 >= prm.coarsest_n;
  return xy && (nz == 0 || (nz % 2 == 0 && nz / 2 >= prm.coarsest_n));
}

size_t esz(bool dbl) { return dbl ? 8 : 4; }

void alloc_fieldset(stc_problem* P, FieldSet& f, const Geom& g, bool dbl) {
  const size_t s = esz(dbl);
  const int N = g.N;
  f.v = dalloc(P, (size_t)(N + 1) * g.F * s);
  f.pbar = dalloc(P, (size_t)(N + 1) * g.C * s);
  f.u = dalloc(P, (size_t)N * g.F * s);
  f.p = dalloc(P, (size_t)N * g.C * s);
}

void check_launch(const char* what) { ck(cudaGetLastError(), what); }

// ---------------------------------------------------------------------------
// NSO building blocks
// ---------------------------------------------------------------------------
// out = sf * f(x) + sr * res  on level l
void nso_residual(stc_problem* P, int l, double sf, double sr, const FieldSet& res, const FieldSet& out,
                  cudaStream_t st, double* sq = nullptr, const double* only_if_undone = nullptr) {
  Level& L = P->lv[l];
  int k = 0;
  dispatch(L.dbl, [&](auto tag) {
    using T = decltype(tag);
    k = launch_nso_residual<T>(L.g, cst_of<T>(L.x), (const T*)L.z, cst_of<T>(res), st_of<T>(out), T(sf), T(sr), st,
                               sq, only_if_undone, P->red, P->lamb3, P->lamb3_bytes);
  });
  count(P, k);
}

// `first_only_if_undone`: the residual in L.tmp is already current unless the
// guarded coarse-grid correction recorded there was undone
void smooth(stc_problem* P, int l, int sweeps, cudaStream_t st, bool timed = false,
            const double* first_only_if_undone = nullptr) {
  Level& L = P->lv[l];
  const int ncol = 1 << L.g.dim;   // parity colours of (i, j[, k])
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < ncol; ++c) {
      // f - res where this colour's cells read it, all from the pre-colour state
      const bool evr = timed && P->ev_used[1] < (int)P->ev_start[1].size();
      if (evr) ck(cudaEventRecordWithFlags(P->ev_start[1][P->ev_used[1]], st, cudaEventRecordExternal), "event");
      int k = 0;
      dispatch(L.dbl, [&](auto tag) {
        using T = decltype(tag);
        k = launch_nso_residual_colour<T>(L.g, cst_of<T>(L.x), (const T*)L.z, cst_of<T>(L.res), st_of<T>(L.tmp), c,
                                          st, s == 0 && c == 0 ? first_only_if_undone : nullptr, P->lamb3,
                                          P->lamb3_bytes);
      });
      if (evr) ck(cudaEventRecordWithFlags(P->ev_stop[1][P->ev_used[1]++], st, cudaEventRecordExternal), "event");
      count(P, k);
      const bool ev = timed && P->ev_used[0] < (int)P->ev_start[0].size();
      if (ev) ck(cudaEventRecordWithFlags(P->ev_start[0][P->ev_used[0]], st, cudaEventRecordExternal), "event");
      int ks = 0;
      dispatch(L.dbl, [&](auto tag) {
        using T = decltype(tag);
        // fp32 mode: fp64 coarsest state and residuals, fp32 per-cell correction solve
        ks = launch_scgs_colour<T>(L.g, st_of<T>(L.x), cst_of<T>(L.tmp), c, !P->dbl, st, P->dlm, P->sc3);
      });
      if (ev) ck(cudaEventRecordWithFlags(P->ev_stop[0][P->ev_used[0]++], st, cudaEventRecordExternal), "event");
      count(P, ks);
    }
}

void restrict_level(stc_problem* P, int l, cudaStream_t st) {
  Level& F = P->lv[l];
  Level& Cc = P->lv[l + 1];
  dispatch(F.dbl, [&](auto tf) {
    using Tf = decltype(tf);
    dispatch(Cc.dbl, [&](auto tc) {
      using Tc = decltype(tc);
      launch_restrict<Tf, Tc>(F.g, Cc.g, cst_of<Tf>(F.x), st_of<Tc>(Cc.x), st_of<Tc>(Cc.old), st);
    });
  });
  count(P, 2);
}

void restrict_residual(stc_problem* P, int l, cudaStream_t st) {
  Level& F = P->lv[l];
  Level& Cc = P->lv[l + 1];
  dispatch(F.dbl, [&](auto tf) {
    using Tf = decltype(tf);
    dispatch(Cc.dbl, [&](auto tc) {
      using Tc = decltype(tc);
      launch_restrict<Tf, Tc>(F.g, Cc.g, cst_of<Tf>(F.tmp), st_of<Tc>(Cc.res), State<Tc>{nullptr, nullptr, nullptr, nullptr},
                              st);
    });
  });
  count(P, 2);
}

void prolong_level(stc_problem* P, int l, cudaStream_t st, const double* undo_if_rose = nullptr) {
  Level& F = P->lv[l];
  Level& Cc = P->lv[l + 1];
  dispatch(F.dbl, [&](auto tf) {
    using Tf = decltype(tf);
    dispatch(Cc.dbl, [&](auto tc) {
      using Tc = decltype(tc);
      launch_prolong_correct<Tf, Tc>(F.g, Cc.g, st_of<Tf>(F.x), cst_of<Tc>(Cc.x), cst_of<Tc>(Cc.old), st,
                                     undo_if_rose);
    });
  });
  count(P, 2);
}

void vcycle_level(stc_problem* P, int l, cudaStream_t st) {
  const int nl = (int)P->lv.size();
  if (l == nl - 1) {
    smooth(P, l, P->prm.coarse_sweeps, st);
    return;
  }
  Level& L = P->lv[l];
  Level& Cc = P->lv[l + 1];
  const bool timed = P->capture_timed && l == 0 && P->counter == &P->graph_launches;
  // guard: norms[0] = ||r^h||_2^2 before the correction, norms[1] after it
  double* norms = P->prm.cgc_guard ? P->dguard + 2 * l : nullptr;
  smooth(P, l, P->prm.pre, st, timed);
  nso_residual(P, l, -1.0, 1.0, L.res, L.tmp, st, norms);  // r^h = res^h - f^h(x^h)
  restrict_level(P, l, st);                                 // x^{2h} = R x^h, kept as XOLD
  restrict_residual(P, l, st);                              // res^{2h} = R r^h
  nso_residual(P, l + 1, 1.0, 1.0, Cc.res, Cc.res, st);     // res^{2h} += f^{2h}(R x^h)
  vcycle_level(P, l + 1, st);
  prolong_level(P, l, st);                                  // x^h += P(x^{2h} - R x^h)
  if (norms) {
    nso_residual(P, l, 1.0, -1.0, L.res, L.tmp, st, norms + 1);   // f^h(x^h) - res^h after it
    prolong_level(P, l, st, norms);                                // undo if the norm rose
    smooth(P, l, P->prm.post, st, timed, norms);
  } else {
    smooth(P, l, P->prm.post, st, timed);
  }
}

void remove_pressure_means(stc_problem* P, cudaStream_t st) {
  Level& L = P->lv[0];
  dispatch(L.dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_remove_mean<T>((T*)L.x.pbar + L.g.C, L.g.N, L.g.C, st);
    launch_remove_mean<T>((T*)L.x.p, L.g.N, L.g.C, st);
  });
  count(P, 2);
}

// ||f(x) - res||_inf of level l into dscal[slot]
void residual_norm(stc_problem* P, int l, int slot, cudaStream_t st) {
  Level& L = P->lv[l];
  nso_residual(P, l, 1.0, -1.0, L.res, L.tmp, st);
  ck(cudaMemsetAsync(P->dscal + slot, 0, sizeof(double), st), "memset");
  const Geom& g = L.g;
  dispatch(L.dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_absmax<T>((const T*)L.tmp.v, (size_t)(g.N + 1) * g.F, P->dscal + slot, P->derr, st);
    launch_absmax<T>((const T*)L.tmp.pbar, (size_t)(g.N + 1) * g.C, P->dscal + slot, P->derr, st);
    launch_absmax<T>((const T*)L.tmp.u, (size_t)g.N * g.F, P->dscal + slot, P->derr, st);
    launch_absmax<T>((const T*)L.tmp.p, (size_t)g.N * g.C, P->dscal + slot, P->derr, st);
  });
  count(P, 4);
}

void copy_state(stc_problem* P, const FieldSet& from, const FieldSet& to, cudaStream_t st) {
  const Geom& g = P->lv[0].g;
  const size_t s = P->ts;
  ck(cudaMemcpyAsync(to.v, from.v, (size_t)(g.N + 1) * g.F * s, cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemcpyAsync(to.pbar, from.pbar, (size_t)(g.N + 1) * g.C * s, cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemcpyAsync(to.u, from.u, (size_t)g.N * g.F * s, cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemcpyAsync(to.p, from.p, (size_t)g.N * g.C * s, cudaMemcpyDeviceToDevice, st), "copy");
}

void enqueue_top_vcycle(stc_problem* P, cudaStream_t st) {
  if (P->prm.lm_adapt) copy_state(P, P->lv[0].x, P->xb, st);   // kept for an undo
  if (P->prm.cgc_guard)
    ck(cudaMemsetAsync(P->dguard, 0, 2 * P->lv.size() * sizeof(double), st), "memset");
  vcycle_level(P, 0, st);
  remove_pressure_means(P, st);
  residual_norm(P, 0, 0, st);
}

// device error flags -> the call's error (no flag: nothing)
void raise_device_errors(int flags) {
  if (flags & DEV_BARRIER_TIMEOUT) fail(STC_ERR_CUDA, "a grid-wide barrier of a 3D sweep timed out");
  if (flags & DEV_TAYLOR_KMAX) fail(STC_ERR_DIVERGED, "Taylor series exceeded taylor_kmax");
  if (flags & DEV_NONFINITE) fail(STC_ERR_DIVERGED, "non-finite value in a residual norm");
}

// Reads a device fp64 scalar (synchronising the stream) and surfaces device
// error flags.  With kmax_rejects (an AO blend trial) a Taylor-order overflow,
// with nonfinite_rejects (an NSO V-cycle under the LM safeguard) a non-finite
// norm, is not an error: the flag is cleared and +inf returned.
double read_scalar(stc_problem* P, int slot, bool kmax_rejects = false, bool nonfinite_rejects = false) {
  // all scalar slots 0..7 come back together (the others stay readable in hscal)
  ck(cudaMemcpyAsync(P->hscal, P->dscal, 8 * sizeof(double), cudaMemcpyDeviceToHost, P->st), "d2h");
  ck(cudaMemcpyAsync(P->herr, P->derr, sizeof(int), cudaMemcpyDeviceToHost, P->st), "d2h");
  ck(cudaStreamSynchronize(P->st), "sync");
  const int rejectable = (kmax_rejects ? DEV_TAYLOR_KMAX : 0) | (nonfinite_rejects ? DEV_NONFINITE : 0);
  if (*P->herr && (*P->herr & ~rejectable) == 0) {
    ck(cudaMemsetAsync(P->derr, 0, sizeof(int), P->st), "memset");
    ck(cudaStreamSynchronize(P->st), "sync");
    return std::numeric_limits<double>::infinity();
  }
  raise_device_errors(*P->herr);
  return P->hscal[slot];
}

// (timed_cycle: with kernel timing on, this cycle runs the graph with events;
// the others run the plain one, so the events perturb one cycle per call)
// captures the V-cycle graph (timed: with the event pairs) if it is not there;
// the plain graph's source is kept for batched launches (a child node)
void ensure_vgraph(stc_problem* P, bool tg) {
  cudaGraphExec_t& ge = tg ? P->vgraph_t : P->vgraph;
  if (!ge) {
    cudaGraph_t graph = nullptr;
    P->graph_launches = 0;
    if (tg) P->ev_used[0] = P->ev_used[1] = 0;
    P->capture_timed = tg;
    P->counter = &P->graph_launches;
    ck(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeRelaxed), "begin capture");
    try {
      enqueue_top_vcycle(P, P->cap);
    } catch (...) {
      P->counter = nullptr;
      P->capture_timed = false;
      cudaStreamEndCapture(P->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    P->counter = nullptr;
    P->capture_timed = false;
    ck(cudaStreamEndCapture(P->cap, &graph), "end capture");
    cudaError_t e = cudaGraphInstantiate(&ge, graph, 0);
    if (!tg && e == cudaSuccess) {
      if (P->vgraph_src) cudaGraphDestroy(P->vgraph_src);
      P->vgraph_src = graph;
      ++P->vgraph_version;
    } else {
      cudaGraphDestroy(graph);
    }
    ck(e, "graph instantiate");
  }
}

double run_vcycle(stc_problem* P, bool nonfinite_rejects = false, bool timed_cycle = false) {
  const bool tg = P->timing && timed_cycle;
  ensure_vgraph(P, tg);
  cudaGraphExec_t& ge = tg ? P->vgraph_t : P->vgraph;
  ck(cudaGraphLaunch(ge, P->st), "graph launch");
  P->launches += P->graph_launches;
  const double f = read_scalar(P, 0, false, nonfinite_rejects);
  for (int kind = 0; tg && kind < 2; ++kind)
    for (int k = 0; k < P->ev_used[kind]; ++k) {
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, P->ev_start[kind][k], P->ev_stop[kind][k]), "event time");
      P->timed_ms[kind] += ms;
      P->timed_launches[kind] += 1;
    }
  return f;
}

void set_lm(stc_problem* P, double lm) {
  P->lm = lm;
  P->hscal[8] = lm;
  ck(cudaMemcpyAsync(P->dlm, P->hscal + 8, sizeof(double), cudaMemcpyHostToDevice, P->st), "h2d");
  ck(cudaStreamSynchronize(P->st), "sync");
}

// One NSO V-cycle under the Levenberg-Marquardt safeguard of Sec. 5 (the FAS
// cycle as the subproblem solver of an LM method): a cycle that raises
// ||f||_inf above f_old, or yields a non-finite norm, is undone and gamma
// (the shift of the smoother's v blocks) is quadrupled.  gamma does not fall
// during one NSO solve (nso_begin halves it back toward its default when the
// next one starts).  The fixed point f = 0 does not depend on gamma.
// Returns the residual of the state kept.
constexpr double kLmMaxRatio = 4096.0;   // largest LM shift relative to its default (4^6)

// *give_up is set when a cycle was undone at the largest shift: the NSO solve
// ends there (unbounded growth left every later cycle undone).
// after one V-cycle that left ||f||_inf = f_new: the LM safeguard's decision
// (Sec. 5) -- a cycle that raised the norm is undone and the shift quadrupled
void lm_decide(stc_problem* P, double f_old, double f_new, double* f, bool* give_up) {
  *give_up = false;
  if (!P->prm.lm_adapt || f_new <= f_old) {
    *f = f_new;
    return;
  }
  copy_state(P, P->xb, P->lv[0].x, P->st);
  ++P->rejected;
  if (P->lm >= kLmMaxRatio * P->lm0) *give_up = true;
  else set_lm(P, std::min(4.0 * P->lm, kLmMaxRatio * P->lm0));
  *f = f_old;
}

double nso_cycle(stc_problem* P, double f_old, bool* give_up) {
  const double f_new = run_vcycle(P, P->prm.lm_adapt != 0);
  double f = f_old;
  lm_decide(P, f_old, f_new, &f, give_up);
  return f;
}

// start of an NSO solve: the LM shift halves back toward its default
void nso_begin(stc_problem* P) {
  if (P->prm.lm_adapt && P->lm > P->lm0) set_lm(P, std::max(P->lm0, 0.5 * P->lm));
}

// ---------------------------------------------------------------------------
// AO / KKT building blocks (finest level)
// ---------------------------------------------------------------------------
void metric_terms(stc_problem* P, const void* rho, cudaStream_t st, double* mterm = nullptr, double* tmp0 = nullptr,
                  double* tmp1 = nullptr) {
  const Geom& g = P->lv[0].g;
  if (!mterm) {
    mterm = P->mterm;
    tmp0 = P->mtmp0;
    tmp1 = P->mtmp1;
  }
  ck(cudaMemsetAsync(mterm, 0, sizeof(double) * (size_t)(g.N + 1) * g.C, st), "memset");
  for (size_t k = 0; k < P->key_steps.size(); ++k) {
    const int s = P->key_steps[k];
    dispatch(P->dbl, [&](auto tag) {
      using T = decltype(tag);
      launch_metric<T>(g, (const T*)rho + (size_t)s * g.C, P->star + k * g.C, P->key_c[k], P->prm.metric_levels,
                       P->prm.metric_sigma0, mterm + (size_t)s * g.C, tmp0, tmp1, st);
    });
  }
  // per keyframe: the difference, then 2D four all-level passes and the level
  // sum, 3D six passes per level; without levels the difference and a scaling
  const int L = P->prm.metric_levels;
  count(P, (long long)P->key_steps.size() * (L > 0 ? (g.dim == 3 ? 1 + 6 * L : 6) : 2));
  check_launch("metric");
}

void forward(stc_problem* P, const void* vel, void* rho, int* K, cudaStream_t st, int* err = nullptr) {
  const Geom& g = P->lv[0].g;
  if (!err) err = P->derr;
  const double thresh = P->prm.taylor_tol * P->rho_scale;
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    if (g.dim == 3)
      ck(launch_taylor_forward3<T>(g, (const T*)vel, (T*)rho, K, thresh, P->prm.taylor_kmax, err, P->adv3, st),
         "taylor forward");
    else
      ck(launch_taylor_forward<T>(g, (const T*)vel, (T*)rho, K, thresh, P->prm.taylor_kmax, err, st),
         "taylor forward");
  });
  count(P, 1);
}

void adjoint(stc_problem* P, const void* vel, const void* rho, const int* K, const void* base, double alpha,
             double beta, void* out, cudaStream_t st, int s_end = 1, void* mu_m1 = nullptr) {
  const Geom& g = P->lv[0].g;
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    if (g.dim == 3)
      ck(launch_taylor_adjoint3<T>(g, (const T*)vel, (const T*)rho, K, P->mterm, (T*)P->mu, (const T*)base, T(alpha),
                                   T(beta), (T*)out, (T*)P->powers, P->prm.taylor_kmax, P->derr, P->adv3, st, s_end,
                                   (T*)mu_m1),
         "taylor adjoint");
    else
      ck(launch_taylor_adjoint<T>(g, (const T*)vel, (const T*)rho, K, P->mterm, (T*)P->mu, (const T*)base, T(alpha),
                                  T(beta), (T*)out, (T*)P->powers, P->prm.taylor_kmax, P->derr, st, s_end,
                                  (T*)mu_m1),
         "taylor adjoint");
  });
  count(P, 1);
}

void project(stc_problem* P, void* fields, int count, cudaStream_t st) {
  const Geom& g = P->lv[0].g;
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    ck(launch_project<T>(g, (T*)fields, count, P->prm.poisson_vcycles, st, (T*)P->pscratch, (const T*)P->dct),
       "project");
  });
  if (count > 0) ::count(P, g.dim == 3 ? project3_launches(g, P->prm.poisson_vcycles) : 1);
}

void prepare_targets(stc_problem* P, cudaStream_t st) {
  Level& L0 = P->lv[0];
  const Geom& g = L0.g;
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_axpby_faces<T>(g, g.N, (const T*)P->vstar, 1.0, (const T*)P->lam, -1.0 / P->prm.K, (T*)L0.z, st);
  });
  for (size_t l = 0; l + 1 < P->lv.size(); ++l) {
    Level& F = P->lv[l];
    Level& Cc = P->lv[l + 1];
    dispatch(F.dbl, [&](auto tf) {
      using Tf = decltype(tf);
      dispatch(Cc.dbl, [&](auto tc) {
        using Tc = decltype(tc);
        launch_restrict_faces<Tf, Tc>(F.g, Cc.g, F.g.N, (const Tf*)F.z, (Tc*)Cc.z, st);
      });
    });
    count(P, 1);
  }
  count(P, 1);
  check_launch("targets");
}

// AO objective of Eq. PO at v* = vel with densities rho (metric terms current):
// 0.5 sum_keys (rho_s - rho*_s)^T C_s (rho_s - rho*_s) + K/2 sum_{i=1}^{N-1} ||w_i - v*_i||^2
// (enqueues the sum into *out, which it zeroes first; mterm: the metric terms of rho)
void enqueue_ao_objective(stc_problem* P, const void* vel, const void* rho, const double* mterm, double* out,
                          cudaStream_t st, const RedScratch& rs) {
  const Geom& g = P->lv[0].g;
  ck(cudaMemsetAsync(out, 0, sizeof(double), st), "memset");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    for (size_t k = 0; k < P->key_steps.size(); ++k) {
      const int s = P->key_steps[k];
      launch_misfit_dot<T>(g, (const T*)rho + (size_t)s * g.C, P->star + k * g.C, mterm + (size_t)s * g.C, out, st,
                           rs);
    }
    launch_diff_sumsq<T>((const T*)P->w + g.F, (const T*)vel + g.F, (size_t)(g.N - 1) * g.F, 0.5 * P->prm.K, out, st,
                         rs);
  });
  count(P, (long long)P->key_steps.size() + (g.N > 1 ? 1 : 0));
  check_launch("ao objective");
}

double ao_objective(stc_problem* P, const void* vel, const void* rho, cudaStream_t st, bool trial = false) {
  enqueue_ao_objective(P, vel, rho, P->mterm, P->dscal + 4, st, P->red);
  return read_scalar(P, 4, trial);
}

// Sec. 5 blend with P->ntrials factors at once (2D): in a round, trial j
// tries a = 2^-(h0 + j) on its own stream and buffers (blend, forward sweep,
// metric terms, objective); the first trial of the round whose objective
// does not exceed J is taken, so the result is the one-at-a-time search's.
// Returns the halvings taken (-1: none) and updates J.
int blend_concurrent(stc_problem* P, double& J, cudaStream_t st) {
  const Geom& g = P->lv[0].g;
  const size_t fb = (size_t)g.F * P->ts;
  double* hval = (double*)P->htrial;
  int* herrs = (int*)(hval + kMaxTrials);
  for (int h0 = 0; h0 <= P->prm.ao_halvings; h0 += P->ntrials) {
    const int nb = std::min(P->ntrials, P->prm.ao_halvings + 1 - h0);
    ck(cudaEventRecord(P->tfork, st), "event");
    for (int j = 0; j < nb; ++j) {
      cudaStream_t s = P->tst[j];
      ck(cudaStreamWaitEvent(s, P->tfork, 0), "wait");
      ck(cudaMemcpyAsync(P->tv[j], P->vstar, fb, cudaMemcpyDeviceToDevice, s), "copy v*_0");
      const double a = std::ldexp(1.0, -(h0 + j));
      dispatch(P->dbl, [&](auto tag) {
        using T = decltype(tag);
        launch_blend_faces<T>(g, g.N - 1, (const T*)P->vstar + g.F, (const T*)P->y + g.F, a, (T*)P->tv[j] + g.F, s);
      });
      count(P, g.N > 1 ? 1 : 0);
      forward(P, P->tv[j], P->trho[j], P->tK[j], s, P->terr + j);
      metric_terms(P, P->trho[j], s, P->tmterm[j], P->ttmp0[j], P->ttmp1[j]);
      enqueue_ao_objective(P, P->tv[j], P->trho[j], P->tmterm[j], P->dtrial + j, s, P->tred[j]);
      ck(cudaEventRecord(P->tdone[j], s), "event");
      ck(cudaStreamWaitEvent(st, P->tdone[j], 0), "wait");
    }
    ck(cudaMemcpyAsync(hval, P->dtrial, nb * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaMemcpyAsync(herrs, P->terr, nb * sizeof(int), cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaMemsetAsync(P->terr, 0, nb * sizeof(int), st), "memset");
    ck(cudaStreamSynchronize(st), "sync");
    // a trial's Taylor-order overflow rejects it (as in read_scalar); any
    // other device error fails the call
    int other = 0;
    for (int j = 0; j < nb; ++j) other |= herrs[j] & ~DEV_TAYLOR_KMAX;
    raise_device_errors(other);
    for (int j = 0; j < nb; ++j) {
      const double Jc = (herrs[j] & DEV_TAYLOR_KMAX) ? std::numeric_limits<double>::infinity() : hval[j];
      if (Jc <= J) {
        std::swap(P->vstar, P->tv[j]);
        std::swap(P->rho, P->trho[j]);
        std::swap(P->K, P->tK[j]);
        std::swap(P->mterm, P->tmterm[j]);
        P->vcand = P->tv[0];
        P->rho_c = P->trho[0];
        P->K_c = P->tK[0];
        J = Jc;
        return h0 + j;
      }
    }
  }
  return -1;
}

void ao(stc_problem* P, int iters, bool warm, cudaStream_t st) {
  Level& L0 = P->lv[0];
  const Geom& g = L0.g;
  const size_t fb = (size_t)g.F * P->ts;
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_ao_init<T>(g, (const T*)L0.x.v, (const T*)P->lam, 1.0 / P->prm.K, (T*)P->w, (T*)P->vstar, warm ? 1 : 0,
                      st);
  });
  count(P, 1);
  P->ao_trace.clear();
  const bool blend = P->prm.ao_halvings >= 0;
  // densities at the starting v* (still valid after a warm start that kept v*)
  if (!(warm && P->rho_at_vstar)) forward(P, P->vstar, P->rho, P->K, st);
  P->rho_at_vstar = true;
  double J = 0.0;
  if (blend && iters > 0) {
    metric_terms(P, P->rho, st);
    J = ao_objective(P, P->vstar, P->rho, st);
  }
  for (int it = 0; it < iters; ++it) {
    // y = Q(w + (dA/dv*)^T mu / K) on steps 1..N-1.  With the blend, mterm
    // already holds C(rho - rho*) of the accepted densities.
    if (!blend) metric_terms(P, P->rho, st);
    adjoint(P, P->vstar, P->rho, P->K, P->w, 1.0, 1.0 / P->prm.K, P->y, st);
    if (g.N > 1) project(P, (char*)P->y + fb, g.N - 1, st);
    if (!blend) {   // plain Alg. 1: v* = y
      if (g.N > 1)
        ck(cudaMemcpyAsync((char*)P->vstar + fb, (char*)P->y + fb, fb * (g.N - 1), cudaMemcpyDeviceToDevice, st),
           "copy v*");
      forward(P, P->vstar, P->rho, P->K, st);
      P->ao_trace.push_back(0);
      continue;
    }
    // Sec. 5 blend: first a = 2^-h whose forward sweep does not raise the objective
    int taken = -1;
    if (P->ntrials > 1) {
      taken = blend_concurrent(P, J, st);
      P->ao_trace.push_back(taken);
      if (taken < 0) break;   // the metric terms of the kept v* are untouched
      continue;
    }
    ck(cudaMemcpyAsync(P->vcand, P->vstar, fb, cudaMemcpyDeviceToDevice, st), "copy v*_0");
    double a = 1.0;
    for (int h = 0; h <= P->prm.ao_halvings; ++h, a *= 0.5) {
      dispatch(P->dbl, [&](auto tag) {
        using T = decltype(tag);
        launch_blend_faces<T>(g, g.N - 1, (const T*)P->vstar + g.F, (const T*)P->y + g.F, a, (T*)P->vcand + g.F,
                              st);
      });
      count(P, g.N > 1 ? 1 : 0);
      forward(P, P->vcand, P->rho_c, P->K_c, st);
      metric_terms(P, P->rho_c, st);
      const double Jc = ao_objective(P, P->vcand, P->rho_c, st, true);
      if (Jc <= J) {
        std::swap(P->vstar, P->vcand);
        std::swap(P->rho, P->rho_c);
        std::swap(P->K, P->K_c);
        J = Jc;
        taken = h;
        break;
      }
    }
    P->ao_trace.push_back(taken);
    if (taken < 0) {
      metric_terms(P, P->rho, st);   // leave the metric terms of the kept v*
      break;
    }
  }
  prepare_targets(P, st);
}

// ||g(v)||^2 into dscal[1]
void kkt(stc_problem* P, cudaStream_t st) {
  Level& L0 = P->lv[0];
  const Geom& g = L0.g;
  // the force branch (u(v) = Q[...], its own buffers and the projection's
  // scratch) runs beside the density branch (forward sweep, metric terms,
  // adjoint sweep: one cluster each) on a second stream
  ck(cudaEventRecord(P->aux_fork, st), "event");
  ck(cudaStreamWaitEvent(P->aux, P->aux_fork, 0), "wait");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_kkt_force_rhs<T>(g, (const T*)L0.x.v, (T*)P->uk, P->aux);
  });
  project(P, P->uk, g.N, P->aux);
  ck(cudaEventRecord(P->aux_join, P->aux), "event");
  forward(P, L0.x.v, P->rho_k, P->Kk, st);
  metric_terms(P, P->rho_k, st);
  adjoint(P, L0.x.v, P->rho_k, P->Kk, nullptr, 0.0, -1.0, P->dens, st);
  ck(cudaStreamWaitEvent(st, P->aux_join, 0), "wait");
  // objective of Eq. opt at v: misfit of rho(v) (dscal[5]) and ||u(v)||^2 (dscal[6])
  ck(cudaMemsetAsync(P->dscal + 5, 0, 2 * sizeof(double), st), "memset");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    for (size_t k = 0; k < P->key_steps.size(); ++k) {
      const int s = P->key_steps[k];
      launch_misfit_dot<T>(g, (const T*)P->rho_k + (size_t)s * g.C, P->star + k * g.C, P->mterm + (size_t)s * g.C,
                           P->dscal + 5, st, P->red);
    }
    launch_sumsq<T>((const T*)P->uk, (size_t)g.N * g.F, P->dscal + 6, st, P->red);
  });
  count(P, (long long)P->key_steps.size() + 1);
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_kkt_grad_rhs<T>(g, (const T*)L0.x.v, (const T*)P->uk, (const T*)P->dens, P->prm.r, (T*)P->gk, st);
  });
  project(P, (char*)P->gk + (size_t)g.F * P->ts, g.N, st);
  ck(cudaMemsetAsync(P->dscal + 1, 0, sizeof(double), st), "memset");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_sumsq<T>((const T*)P->gk, (size_t)(g.N + 1) * g.F, P->dscal + 1, st, P->red);
  });
  count(P, 3);
  check_launch("kkt");
}

template <class T>
__global__ void lambda_update_kernel(size_t n, size_t skip, T* lam, const T* __restrict__ v, const T* __restrict__ vs,
                                     double kb) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    if (e >= skip) lam[e] += T(kb) * (v[e] - vs[e]);
}

// Alg. 3's density test (max |rho - rho^last| into dscal[2], rho^last <- rho)
// and, unless the AL fallback holds it back, the multiplier update.
void admm_update(stc_problem* P, cudaStream_t st, bool update_lambda = true) {
  Level& L0 = P->lv[0];
  const Geom& g = L0.g;
  ck(cudaMemsetAsync(P->dscal + 2, 0, sizeof(double), st), "memset");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_absdiff_max_copy<T>((const T*)P->rho, (T*)P->rho_last, (size_t)(g.N + 1) * g.C, P->dscal + 2, st);
    if (update_lambda) {
      const size_t n = (size_t)g.N * g.F;
      unsigned nb = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
      lambda_update_kernel<T><<<nb, 256, 0, st>>>(n, (size_t)g.F, (T*)P->lam, (const T*)L0.x.v,
                                                   (const T*)P->vstar, P->prm.K * P->prm.beta);
    }
  });
  count(P, update_lambda ? 2 : 1);
  check_launch("admm update");
}

void reset_state(stc_problem* P) {
  for (Level& L : P->lv) {
    const Geom& g = L.g;
    const size_t s = esz(L.dbl);
    FieldSet* sets[3] = {&L.x, &L.res, &L.tmp};
    for (FieldSet* f : sets) {
      ck(cudaMemsetAsync(f->v, 0, (size_t)(g.N + 1) * g.F * s, P->st), "memset");
      ck(cudaMemsetAsync(f->pbar, 0, (size_t)(g.N + 1) * g.C * s, P->st), "memset");
      ck(cudaMemsetAsync(f->u, 0, (size_t)g.N * g.F * s, P->st), "memset");
      ck(cudaMemsetAsync(f->p, 0, (size_t)g.N * g.C * s, P->st), "memset");
    }
  }
  const Geom& g = P->lv[0].g;
  ck(cudaMemcpyAsync(P->lv[0].x.v, P->v0, (size_t)g.F * P->ts, cudaMemcpyDeviceToDevice, P->st), "v0");
  ck(cudaMemsetAsync(P->lam, 0, (size_t)g.N * g.F * P->ts, P->st), "memset");
  P->rho_at_vstar = false;
  P->lm0 = g.lm;
  P->rejected = 0;
  set_lm(P, P->lm0);
}

// ---------------------------------------------------------------------------
// field access
// ---------------------------------------------------------------------------
struct FieldRef {
  void* ptr = nullptr;
  size_t count = 0;
  int kind = 0;  // 0: level type, 1: fp64
  bool dbl = false;
};

// buffers of the forward simulation and its adjoint, allocated at first use
// (a control problem that never simulates does not hold them)
void sim_alloc(stc_problem* P) {
  if (P->sim_gu) return;
  const Geom& g = P->lv[0].g;
  const size_t ts = P->ts, N = g.N;
  P->sim_gu = dalloc(P, N * g.F * ts);
  P->sim_a0 = dalloc(P, g.F * ts);
  P->sim_l0 = dalloc(P, g.C * ts);
  P->sim_aN = dalloc(P, g.F * ts);
  P->sim_w1 = dalloc(P, g.F * ts);
  P->sim_w2 = dalloc(P, g.F * ts);
  P->sim_w3 = dalloc(P, g.F * ts);
  P->sim_grho = (double*)dalloc(P, (N + 1) * g.C * sizeof(double));
}

// max |a - b| over the interior of a face slab into dscal[slot], b = a; and
// max |b| into dscal[slot + 1]; returns the pair after a synchronising read
std::pair<double, double> step_change(stc_problem* P, const void* a, void* b, cudaStream_t st, int slot) {
  const Geom& g = P->lv[0].g;
  ck(cudaMemsetAsync(P->dscal + slot, 0, 2 * sizeof(double), st), "memset");
  dispatch(P->dbl, [&](auto tag) {
    using T = decltype(tag);
    launch_absdiff_max_copy<T>((const T*)a, (T*)b, (size_t)g.F, P->dscal + slot, st);
    launch_absmax<T>((const T*)b, (size_t)g.F, P->dscal + slot + 1, P->derr, st);
  });
  count(P, 2);
  const double d = read_scalar(P, slot);
  return {d, P->hscal[slot + 1]};
}

// Convergence of the (transposed) Picard iteration: the change d at most tol *
// max|x|, or -- the rounding floor of the state type -- d no longer halving
// after 8 iterations while within 100 tol * max|x| (the iteration map is a
// fixed linear-plus-Adv map whose change cannot fall below its rounding).
bool picard_done(double d, double xmax, double tol, int it, double* prev) {
  const double ref = tol * std::max(xmax, 1e-300);
  const bool done = d <= ref || (it >= 8 && d >= 0.5 * *prev && d <= 100.0 * ref);
  *prev = d;
  return done;
}

// v_{t+1} from v_t and u_t: Picard v <- Q[v_t + dt (u_t - Adv(v))] until the
// change is at most tol * max|v|; returns the iterations used
int picard_step(stc_problem* P, int t, double tol, int max_iter) {
  const Geom& g = P->lv[0].g;
  const size_t fb = (size_t)g.F * P->ts;
  char* v = (char*)P->lv[0].x.v;
  const char* u = (const char*)P->lv[0].x.u;
  ck(cudaMemcpyAsync(v + (t + 1) * fb, v + t * fb, fb, cudaMemcpyDeviceToDevice, P->st), "copy");
  double prev = std::numeric_limits<double>::infinity();
  for (int it = 1; it <= max_iter; ++it) {
    dispatch(P->dbl, [&](auto tag) {
      using T = decltype(tag);
      launch_picard_rhs<T>(g, (const T*)(v + t * fb), (const T*)(u + t * fb), (const T*)(v + (t + 1) * fb), g.dt,
                           (T*)P->sim_w1, P->st);
    });
    count(P, 1);
    project(P, P->sim_w1, 1, P->st);
    const auto dm = step_change(P, P->sim_w1, v + (t + 1) * fb, P->st, 6);
    if (!(dm.first == dm.first)) fail(STC_ERR_DIVERGED, "non-finite velocity in the implicit step");
    if (picard_done(dm.first, dm.second, tol, it, &prev)) return it;
  }
  fail(STC_ERR_NOT_CONVERGED, "implicit Navier-Stokes step: Picard iteration did not converge (change " +
                                  std::to_string(prev) + ")");
  return max_iter;
}

// z = Q[a - dt dAdv(v_{t+1})^T z] (the transposed step), z into sim_w2
int picard_adjoint_step(stc_problem* P, int t, const void* a, double tol, int max_iter) {
  const Geom& g = P->lv[0].g;
  const size_t fb = (size_t)g.F * P->ts;
  const char* v = (const char*)P->lv[0].x.v;
  ck(cudaMemsetAsync(P->sim_w2, 0, fb, P->st), "memset");
  double prev = std::numeric_limits<double>::infinity();
  for (int it = 1; it <= max_iter; ++it) {
    dispatch(P->dbl, [&](auto tag) {
      using T = decltype(tag);
      launch_picard_adj_rhs<T>(g, (const T*)(v + (t + 1) * fb), (const T*)a, (const T*)P->sim_w2, g.dt,
                               (T*)P->sim_w3, P->st);
    });
    count(P, 1);
    project(P, P->sim_w3, 1, P->st);
    const auto dm = step_change(P, P->sim_w3, P->sim_w2, P->st, 6);
    if (!(dm.first == dm.first)) fail(STC_ERR_DIVERGED, "non-finite value in the transposed implicit step");
    if (picard_done(dm.first, dm.second, tol, it, &prev)) return it;
  }
  fail(STC_ERR_NOT_CONVERGED, "transposed implicit step: iteration did not converge (change " +
                                  std::to_string(prev) + ")");
  return max_iter;
}

FieldRef field_ref(stc_problem* P, int field, int level) {
  const int nl = (int)P->lv.size();
  if (level < 0 || level >= nl) fail(STC_ERR_INVALID_ARG, "level out of range");
  Level& L = P->lv[level];
  const Geom& g = L.g;
  const size_t N = g.N;
  FieldRef r;
  r.dbl = L.dbl;
  auto set4 = [&](const FieldSet& f, int which) {
    switch (which) {
      case 0: r.ptr = f.v; r.count = (N + 1) * g.F; break;
      case 1: r.ptr = f.pbar; r.count = (N + 1) * g.C; break;
      case 2: r.ptr = f.u; r.count = N * g.F; break;
      default: r.ptr = f.p; r.count = N * g.C; break;
    }
  };
  if (field >= STC_FIELD_V && field <= STC_FIELD_P) {
    set4(L.x, field - STC_FIELD_V);
    return r;
  }
  if (field >= STC_FIELD_RES_V && field <= STC_FIELD_RES_P) {
    set4(L.tmp, field - STC_FIELD_RES_V);
    return r;
  }
  if (field >= STC_FIELD_RES_IN_V && field <= STC_FIELD_RES_IN_P) {
    set4(L.res, field - STC_FIELD_RES_IN_V);
    return r;
  }
  if (field >= STC_FIELD_XOLD_V && field <= STC_FIELD_XOLD_P) {
    if (level == 0) fail(STC_ERR_INVALID_ARG, "XOLD exists on coarse levels only");
    set4(L.old, field - STC_FIELD_XOLD_V);
    return r;
  }
  if (field == STC_FIELD_Z) {
    r.ptr = L.z;
    r.count = N * g.F;
    return r;
  }
  if (level != 0) fail(STC_ERR_INVALID_ARG, "field exists on the finest level only");
  r.dbl = P->dbl;
  switch (field) {
    case STC_FIELD_VSTAR: r.ptr = P->vstar; r.count = N * g.F; break;
    case STC_FIELD_LAMBDA: r.ptr = P->lam; r.count = N * g.F; break;
    case STC_FIELD_RHO: r.ptr = P->rho; r.count = (N + 1) * g.C; break;
    case STC_FIELD_MU: r.ptr = P->mu; r.count = N * g.C; break;
    case STC_FIELD_W: r.ptr = P->w; r.count = N * g.F; break;
    case STC_FIELD_Y: r.ptr = P->y; r.count = N * g.F; break;
    case STC_FIELD_KKT_U: r.ptr = P->uk; r.count = N * g.F; break;
    case STC_FIELD_KKT_G: r.ptr = P->gk; r.count = (N + 1) * g.F; break;
    case STC_FIELD_MTERM: r.ptr = P->mterm; r.count = (N + 1) * g.C; r.kind = 1; break;
    case STC_FIELD_SIM_GRAD_RHO: sim_alloc(P); r.ptr = P->sim_grho; r.count = (N + 1) * g.C; r.kind = 1; break;
    case STC_FIELD_SIM_GRAD_U: sim_alloc(P); r.ptr = P->sim_gu; r.count = N * g.F; break;
    case STC_FIELD_SIM_ADJ_V0: sim_alloc(P); r.ptr = P->sim_a0; r.count = g.F; break;
    case STC_FIELD_SIM_ADJ_RHO0: sim_alloc(P); r.ptr = P->sim_l0; r.count = g.C; break;
    case STC_FIELD_SIM_ADJ_VN: sim_alloc(P); r.ptr = P->sim_aN; r.count = g.F; break;
    default: fail(STC_ERR_INVALID_ARG, "unknown field id");
  }
  return r;
}

void copy_out(stc_problem* P, const FieldRef& r, double* out) {
  if (r.kind == 1 || r.dbl) {
    ck(cudaMemcpyAsync(out, r.ptr, r.count * sizeof(double), cudaMemcpyDeviceToHost, P->st), "d2h");
    ck(cudaStreamSynchronize(P->st), "sync");
    return;
  }
  std::vector<float> tmp(r.count);
  ck(cudaMemcpyAsync(tmp.data(), r.ptr, r.count * sizeof(float), cudaMemcpyDeviceToHost, P->st), "d2h");
  ck(cudaStreamSynchronize(P->st), "sync");
  for (size_t e = 0; e < r.count; ++e) out[e] = (double)tmp[e];
}

void copy_in(stc_problem* P, const FieldRef& r, const double* in) {
  if (r.kind == 1 || r.dbl) {
    ck(cudaMemcpyAsync(r.ptr, in, r.count * sizeof(double), cudaMemcpyHostToDevice, P->st), "h2d");
    ck(cudaStreamSynchronize(P->st), "sync");
    return;
  }
  std::vector<float> tmp(r.count);
  for (size_t e = 0; e < r.count; ++e) tmp[e] = (float)in[e];
  ck(cudaMemcpyAsync(r.ptr, tmp.data(), r.count * sizeof(float), cudaMemcpyHostToDevice, P->st), "h2d");
  ck(cudaStreamSynchronize(P->st), "sync");
}

template <class F>
stc_status guarded(stc_problem* P, F&& f) {
  if (P && P->broken) {
    g_last_error = "problem is unusable after an earlier CUDA error";
    return STC_ERR_CUDA;
  }
  try {
    f();
    return STC_OK;
  } catch (const StcError& e) {
    g_last_error = e.msg;
    if (P && e.code == STC_ERR_CUDA) P->broken = true;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return STC_ERR_OOM;
  } catch (...) {
    g_last_error = "unexpected error";
    return STC_ERR_CUDA;
  }
}

bool params_valid(const stc_params& prm) {
  return !(prm.nx < 2 || prm.ny < 2 || prm.num_steps < 1 || !(prm.dt > 0) || !(prm.r > 0) || !(prm.K > 0) ||
      prm.precision < 0 || prm.precision > 1 || prm.ao_iters < 0 || prm.pre < 0 || prm.post < 0 ||
      prm.coarse_sweeps < 0 || prm.coarsest_n < 2 || !(prm.taylor_tol > 0) || prm.taylor_kmax < 1 ||
      prm.taylor_kmax > 256 || prm.max_vcycles < 0 || prm.metric_levels < 0 || prm.metric_levels > 12 ||
      !(prm.scgs_omega > 0) || prm.poisson_vcycles < 1 || prm.ao_halvings < -1 || prm.ao_halvings > 60 ||
      prm.cgc_guard < 0 || prm.cgc_guard > 1 || prm.lm_adapt < 0 || prm.lm_adapt > 1 ||
      prm.al_threshold != prm.al_threshold || prm.time_coarsen < 0 || prm.time_coarsen > 1 || prm.nz < 0 ||
      prm.nz == 1 || prm.boundary < 0 || prm.boundary > 1 || prm.scgs_cta_cells < -1 || prm.ao_trials < 1 || prm.ao_trials > kMaxTrials ||
      prm.k_adapt < 0 || prm.k_adapt > 1 ||
      (prm.boundary == 1 && (prm.nz == 0 || prm.nx % 2 || prm.ny % 2 || prm.nz % 2)));
}

// Device bytes that stc_create_problem plus stc_set_keyframes(nkeys) allocate:
// the same list of buffers as the allocations below, without allocating
// (the serving admission test).  Must be kept in step with them.
// blend trials run at once: 2D with the blend on; 3D sweeps share one scratch
int ao_trial_count(const stc_params& prm) {
  return (prm.nz == 0 && prm.ao_halvings >= 0) ? std::min(prm.ao_trials, std::min(kMaxTrials, prm.ao_halvings + 1))
                                               : 1;
}

size_t plan_bytes(const stc_params& prm, int nkeys) {
  auto b = [](size_t n) { return n == 0 ? (size_t)16 : n; };
  const bool dbl = prm.precision == 1;
  const size_t ts = dbl ? 8 : 4;
  const size_t N = (size_t)prm.num_steps;
  struct Dim { int nx, ny, nz, N; };
  std::vector<Dim> dims{{prm.nx, prm.ny, prm.nz, prm.num_steps}};
  int nx = prm.nx, ny = prm.ny, nz = prm.nz, Nl = prm.num_steps;
  while (can_halve(prm, nx, ny, nz)) {
    nx /= 2;
    ny /= 2;
    nz /= 2;
    if (prm.time_coarsen && Nl % 2 == 0) Nl /= 2;
    dims.push_back({nx, ny, nz, Nl});
  }
  auto faces = [](int x, int y, int z) {
    return z > 0 ? (size_t)z * y * (x + 1) + (size_t)z * (y + 1) * x + (size_t)(z + 1) * y * x
                 : (size_t)y * (x + 1) + (size_t)(y + 1) * x;
  };
  auto cells = [](int x, int y, int z) { return (size_t)x * y * (z > 0 ? z : 1); };
  auto fieldset = [&](size_t F, size_t C, size_t s, size_t Nl_) {
    return b((Nl_ + 1) * F * s) + b((Nl_ + 1) * C * s) + b(Nl_ * F * s) + b(Nl_ * C * s);
  };
  size_t total = 0;
  for (size_t l = 0; l < dims.size(); ++l) {
    const size_t F = faces(dims[l].nx, dims[l].ny, dims[l].nz), C = cells(dims[l].nx, dims[l].ny, dims[l].nz);
    const size_t Nl_ = (size_t)dims[l].N;
    const size_t s = (dbl || (l > 0 && l == dims.size() - 1)) ? 8 : 4;
    total += 3 * fieldset(F, C, s, Nl_) + (l > 0 ? fieldset(F, C, s, Nl_) : 0) + b(Nl_ * F * s);
  }
  const size_t F = faces(prm.nx, prm.ny, prm.nz), C = cells(prm.nx, prm.ny, prm.nz);
  total += 3 * b((N + 1) * C * ts) + b(N * C * ts) + 2 * b(N * F * ts) + b((N + 1) * C * ts) + b(N * 4) +
           b(2 * dims.size() * 8) + b(8) + (prm.lm_adapt ? fieldset(F, C, ts, N) : 0) +
           (prm.k_adapt ? b((N + 1) * F * ts) : 0) + 4 * b(N * F * ts) +
           2 * b((N + 1) * F * ts) + b((size_t)prm.taylor_kmax * C * ts) + b(F * ts) + 2 * b(N * 4) +
           b((N + 1) * C * 8) + b(C * 8) + b(metric_tmp1_doubles(C, prm.metric_levels) * 8) + b(16 * 8) + b(4);
  if (nkeys > 0) total += b((size_t)nkeys * C * 8);
  total += b(red_capacity(make_geom(prm, prm.nx, prm.ny, prm.nz, 1.0 / prm.nx, prm.num_steps, prm.dt)) * 8) + b(4);
  const int nt = ao_trial_count(prm);
  if (nt > 1) total += (size_t)nt * (b(kReduceMaxBlocks * 8) + b(4));
  if (nt > 1)
    total += (size_t)(nt - 1) * (b(N * F * ts) + b((N + 1) * C * ts) + b(N * 4) + b(C * 8) +
                                 b(metric_tmp1_doubles(C, prm.metric_levels) * 8)) +
             (size_t)nt * b((N + 1) * C * 8) + b(kMaxTrials * 4) + b(kMaxTrials * 8);
  Geom g0 = make_geom(prm, prm.nx, prm.ny, prm.nz, 1.0 / prm.nx, prm.num_steps, prm.dt);
  if (project_dct_fits(g0, ts)) total += b(project_dct_elems(g0) * ts);
  if (g0.dim == 3) {
    total += b(advect3_scratch_bytes(g0, ts)) + b(project3_scratch_elems(g0, (int)N + 1) * ts) +
             b(scgs3_thomas_scratch_bytes(g0, ts));
    const Dim& dc = dims.back();
    const Geom gc = make_geom(prm, dc.nx, dc.ny, dc.nz, 1.0 / dc.nx, dc.N, prm.dt);
    const size_t lb = lamb3_scratch_bytes_max(g0, ts, gc, dims.size() > 1 ? 8 : ts);
    if (lb > 0) total += b(lb);
  } else if (project_needs_scratch(g0, ts)) {
    total += b((N + 1) * project_smem(g0, ts));
  }
  return total;
}

void free_problem(stc_problem* P) {
  if (!P) return;
  if (P->vgraph) cudaGraphExecDestroy(P->vgraph);
  if (P->vgraph_t) cudaGraphExecDestroy(P->vgraph_t);
  if (P->vgraph_src) cudaGraphDestroy(P->vgraph_src);
  for (int kind = 0; kind < 2; ++kind) {
    for (cudaEvent_t e : P->ev_start[kind]) cudaEventDestroy(e);
    for (cudaEvent_t e : P->ev_stop[kind]) cudaEventDestroy(e);
  }
  for (void* p : P->allocs) cudaFree(p);
  if (P->hscal) cudaFreeHost(P->hscal);
  if (P->herr) cudaFreeHost(P->herr);
  if (P->cap) cudaStreamDestroy(P->cap);
  for (int j = 0; j < kMaxTrials; ++j) {
    if (P->tst[j]) cudaStreamDestroy(P->tst[j]);
    if (P->tdone[j]) cudaEventDestroy(P->tdone[j]);
  }
  if (P->tfork) cudaEventDestroy(P->tfork);
  if (P->aux) cudaStreamDestroy(P->aux);
  if (P->aux_fork) cudaEventDestroy(P->aux_fork);
  if (P->aux_join) cudaEventDestroy(P->aux_join);
  if (P->htrial) cudaFreeHost(P->htrial);
  delete P;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// the V-cycle graphs (captured again at the next cycle)
void drop_vgraphs(stc_problem* p) {
  for (cudaGraphExec_t* ge : {&p->vgraph, &p->vgraph_t})
    if (*ge) {
      ck(cudaGraphExecDestroy(*ge), "graph destroy");
      *ge = nullptr;
    }
  if (p->vgraph_src) {
    cudaGraphDestroy(p->vgraph_src);
    p->vgraph_src = nullptr;
  }
}

// the ADMM penalty of every level and the multiplier step; the V-cycle graphs
// carry K/r in their kernel arguments and are captured again at the next cycle
void set_penalty_impl(stc_problem* p, double K, double beta) {
  ck(cudaStreamSynchronize(p->st), "sync");
  p->prm.K = K;
  p->prm.beta = beta;
  for (Level& L : p->lv) {
    L.g.a = K / p->prm.r;
    set_fp32_copies(L.g);
  }
  drop_vgraphs(p);
}

// Residual balancing of the ADMM penalty (stc_params.k_adapt; the paper keeps
// K fixed): with the primal residual r_p = ||v - v*|| and the dual residual
// r_d = K ||v - v_prev|| over steps 1..N-1 (v_prev: the previous iteration's
// v), K doubles when r_p > 10 r_d and halves when r_d > 10 r_p, within 2^+-10
// of its value at the start of the solve.  first: only v_prev is recorded.
constexpr double kAdaptMu = 10.0, kAdaptTau = 2.0, kAdaptRange = 1024.0;

void adapt_penalty(stc_problem* P, bool first, double K0) {
  const Geom& g = P->lv[0].g;
  const size_t fb = (size_t)(g.N + 1) * g.F * P->ts;
  if (!first && g.N > 1) {
    ck(cudaMemsetAsync(P->dscal + 10, 0, 2 * sizeof(double), P->st), "memset");
    dispatch(P->dbl, [&](auto tag) {
      using T = decltype(tag);
      const size_t n = (size_t)(g.N - 1) * g.F;
      launch_diff_sumsq<T>((const T*)P->lv[0].x.v + g.F, (const T*)P->vstar + g.F, n, 1.0, P->dscal + 10, P->st,
                           P->red);
      launch_diff_sumsq<T>((const T*)P->lv[0].x.v + g.F, (const T*)P->vprev + g.F, n, 1.0, P->dscal + 11, P->st,
                           P->red);
    });
    count(P, 2);
    ck(cudaMemcpyAsync(P->hscal + 10, P->dscal + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, P->st), "d2h");
    ck(cudaStreamSynchronize(P->st), "sync");
    const double K = P->prm.K;
    const double rp = std::sqrt(P->hscal[10]), rd = K * std::sqrt(P->hscal[11]);
    double Kn = K;
    if (rp > kAdaptMu * rd) Kn = K * kAdaptTau;
    else if (rd > kAdaptMu * rp) Kn = K / kAdaptTau;
    Kn = std::min(std::max(Kn, K0 / kAdaptRange), K0 * kAdaptRange);
    if (Kn != K) set_penalty_impl(P, Kn, P->prm.beta);
  }
  ck(cudaMemcpyAsync(P->vprev, P->lv[0].x.v, fb, cudaMemcpyDeviceToDevice, P->st), "copy");
}

// ---------------------------------------------------------------------------
// stc_solve as resumable phases (Alg. 3): begin; then per ADMM iteration the
// head (Alg. 1 and the NSO residual), NSO V-cycles until the tolerance (one per
// call of solve_cycle_done after a V-cycle ran), and the tail (KKT metric,
// multiplier update, stopping tests).  stc_solve runs them in a loop; a
// serving step runs the V-cycles of many problems in one graph launch.
// ---------------------------------------------------------------------------
void solve_begin(stc_problem* p, double tol, int max_admm) {
  SolveRun& S = p->run;
  S = SolveRun{};
  std::memset(&S.rep, 0, sizeof(S.rep));
  S.rep.seconds_to_1e4 = -1.0;
  S.rep.seconds_to_1e2 = S.rep.seconds_to_1e3 = S.rep.seconds_to_1e6 = -1.0;
  S.rep.seconds_to_density_stop = -1.0;
  S.rep.K_final = p->prm.K;
  S.tol = tol;
  S.max_admm = max_admm;
  S.t0 = std::chrono::steady_clock::now();
  S.K0 = p->prm.K;
  p->solve_hist.clear();
  reset_state(p);
  const Geom& g = p->lv[0].g;
  S.eps_admm = p->prm.eps_admm < 0 ? p->rho_scale / 100.0 : p->prm.eps_admm;
  // rho^last = uncontrolled densities; KKT denominator at the start
  kkt(p, p->st);
  S.g0 = std::sqrt(read_scalar(p, 1));
  S.J_prev = p->hscal[5] + 0.5 * p->prm.r * p->hscal[6];   // objective at v_start
  ck(cudaMemcpyAsync(p->rho_last, p->rho_k, (size_t)(g.N + 1) * g.C * p->ts, cudaMemcpyDeviceToDevice, p->st),
     "copy");
  p->fscale = -1.0;
  S.phase = max_admm > 0 ? 0 : 2;
}

// Alg. 1 (warm-started after the first iteration), the NSO residual, the start of the NSO solve
void solve_head(stc_problem* p) {
  SolveRun& S = p->run;
  ao(p, p->prm.ao_iters, S.it > 0, p->st);
  residual_norm(p, 0, 0, p->st);
  S.f = read_scalar(p, 0);
  if (p->fscale < 0) p->fscale = S.f;
  S.cycles = 0;
  S.give_up = false;
  nso_begin(p);
  S.phase = 1;
}

// at least one V-cycle per ADMM iteration, then until the NSO tolerance or the cap
bool solve_wants_cycle(const stc_problem* p) {
  const SolveRun& S = p->run;
  return S.phase == 1 && (S.cycles < 1 || S.f > p->prm.eps_stfas * p->fscale) && S.cycles < p->prm.max_vcycles &&
         !S.give_up;
}

void solve_cycle_done(stc_problem* p, double f_new) {
  SolveRun& S = p->run;
  lm_decide(p, S.f, f_new, &S.f, &S.give_up);
  ++S.cycles;
}

// KKT metric, AL-fallback decision, multiplier update, penalty balancing, stopping tests
void solve_tail(stc_problem* p) {
  SolveRun& S = p->run;
  stc_report& rep = S.rep;
  const stc_params& prm = p->prm;
  kkt(p, p->st);
  const double gn = std::sqrt(read_scalar(p, 1));
  const double J = p->hscal[5] + 0.5 * prm.r * p->hscal[6];
  // Sec. 5 AL fallback: hold lambda while the objective still falls by more
  // than al_threshold * |J| per iteration (al_threshold < 0: plain Alg. 3)
  const bool update = prm.al_threshold < 0 || (S.J_prev - J) <= prm.al_threshold * std::fabs(S.J_prev);
  S.J_prev = J;
  admm_update(p, p->st, update);   // drho test + lambda update (lambda unused if we stop)
  const double drho = read_scalar(p, 2);
  const double K_used = prm.K;
  if (prm.k_adapt && update) {
    adapt_penalty(p, !S.have_prev, S.K0);
    S.have_prev = true;
  }
  rep.objective = J;
  if (update) ++rep.lambda_updates;
  rep.admm_iters = S.it + 1;
  rep.vcycles += S.cycles;
  rep.rejected_vcycles = p->rejected;
  rep.lm_shift = p->lm;
  rep.kkt_abs = gn;
  rep.kkt_rel = S.g0 > 0 ? gn / S.g0 : 0.0;
  rep.f_inf = S.f;
  rep.drho = drho;
  const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
  p->solve_hist.insert(p->solve_hist.end(), {rep.kkt_rel, el, K_used});
  if (rep.kkt_rel <= 1e-2 && rep.seconds_to_1e2 < 0) rep.seconds_to_1e2 = el;
  if (rep.kkt_rel <= 1e-3 && rep.seconds_to_1e3 < 0) rep.seconds_to_1e3 = el;
  if (rep.kkt_rel <= 1e-4 && rep.seconds_to_1e4 < 0) rep.seconds_to_1e4 = el;
  if (rep.kkt_rel <= 1e-6 && rep.seconds_to_1e6 < 0) rep.seconds_to_1e6 = el;
  rep.K_final = K_used;
  if (drho < p->rho_scale / 100.0 && rep.density_stop_iter == 0) {
    rep.density_stop_iter = S.it + 1;
    rep.seconds_to_density_stop = el;
  }
  ++S.it;
  if (rep.kkt_rel <= S.tol || drho < S.eps_admm) {
    S.converged = true;
    S.phase = 2;
  } else {
    S.phase = S.it < S.max_admm ? 0 : 2;
  }
  if (S.phase == 2) {
    ck(cudaStreamSynchronize(p->st), "sync");
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
  }
}

extern "C" {

void stc_default_params(stc_params* p, int nx, int ny, int num_steps) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->num_steps = num_steps;
  p->dt = num_steps > 0 ? 1.0 / num_steps : 0.0;
  p->r = 1e-3;
  p->K = 1.0;
  p->beta = 1.0;
  p->precision = 0;
  p->ao_iters = 2;
  p->pre = 2;
  p->post = 2;
  p->coarse_sweeps = 10;
  p->coarsest_n = 4;
  p->taylor_tol = 1e-5;
  p->taylor_kmax = 64;
  p->eps_stfas = 1e-5;
  p->eps_admm = -1.0;
  p->max_vcycles = 20;
  p->metric_levels = 0;
  p->metric_sigma0 = 1.0;
  p->scgs_omega = 0.8;
  p->lm_shift = -1.0;
  p->poisson_vcycles = 8;
  p->self_advection = 1;
  p->ao_halvings = 8;
  p->cgc_guard = 1;
  p->lm_adapt = 1;
  p->al_threshold = -1.0;
  p->time_coarsen = 0;
  p->nz = 0;
  p->boundary = 0;
  p->scgs_cta_cells = -1;
  p->ao_trials = 4;
  p->k_adapt = 0;
}

const char* stc_last_error(void) { return g_last_error.c_str(); }

stc_status stc_create_problem(const stc_params* params, const double* rho0, const double* v0, void* cuda_stream,
                              stc_problem** out) {
  if (!params || !rho0 || !out) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const stc_params& prm = *params;
  if (!params_valid(prm)) {
    g_last_error = "invalid parameters";
    return STC_ERR_INVALID_ARG;
  }
  stc_problem* P = new (std::nothrow) stc_problem();
  if (!P) {
    g_last_error = "host allocation failed";
    return STC_ERR_OOM;
  }
  P->prm = prm;
  P->st = (cudaStream_t)cuda_stream;
  P->dbl = prm.precision == 1;
  P->ts = P->dbl ? 8 : 4;
  stc_status s = guarded(nullptr, [&]() {
    // hierarchy: halve while both even and the halves stay >= coarsest_n (in
    // space, Sec. 4.2); with time_coarsen each level whose N is even also
    // hands the next one N/2 steps of 2 dt
    int nx = prm.nx, ny = prm.ny, nz = prm.nz, Nl = prm.num_steps;
    double h = 1.0 / prm.nx, dtl = prm.dt;
    std::vector<Geom> geoms;
    geoms.push_back(make_geom(prm, nx, ny, nz, h, Nl, dtl));
    while (can_halve(prm, nx, ny, nz)) {
      nx /= 2;
      ny /= 2;
      nz /= 2;
      h *= 2.0;
      if (prm.time_coarsen && Nl % 2 == 0) {
        Nl /= 2;
        dtl *= 2.0;
      }
      geoms.push_back(make_geom(prm, nx, ny, nz, h, Nl, dtl));
    }
    const Geom& g0 = geoms[0];
    const bool d3 = g0.dim == 3;
    if (!d3 && !advect_supported(g0)) fail(STC_ERR_UNSUPPORTED, "grid too large for the on-chip advection sweep");
    if (!d3 && !project_supported(g0, P->ts)) fail(STC_ERR_UNSUPPORTED, "grid too large for the on-chip projection");
    if (d3 && !project3_supported(g0)) fail(STC_ERR_UNSUPPORTED, "coarsest projection level above 512 cells");
    int dev = 0;
    ck(cudaGetDevice(&dev), "get device");
    int smem_optin = 0;
    ck(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
    if (!d3 && ((int)advect_smem_adjoint(g0, P->ts) > smem_optin ||
                (!project_needs_scratch(g0, P->ts) && (int)project_smem(g0, P->ts) > smem_optin)))
      fail(STC_ERR_UNSUPPORTED, "shared memory of this device too small for the grid");
    ck(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking), "stream");
    ck(cudaStreamCreateWithFlags(&P->aux, cudaStreamNonBlocking), "stream");
    ck(cudaEventCreateWithFlags(&P->aux_fork, cudaEventDisableTiming), "event");
    ck(cudaEventCreateWithFlags(&P->aux_join, cudaEventDisableTiming), "event");
    const int N = prm.num_steps;
    for (size_t l = 0; l < geoms.size(); ++l) {
      Level L;
      L.g = geoms[l];
      L.dbl = P->dbl || (l > 0 && l == geoms.size() - 1);   // fp64 coarsest level (precision policy)
      alloc_fieldset(P, L.x, L.g, L.dbl);
      alloc_fieldset(P, L.res, L.g, L.dbl);
      alloc_fieldset(P, L.tmp, L.g, L.dbl);
      if (l > 0) alloc_fieldset(P, L.old, L.g, L.dbl);
      L.z = dalloc(P, (size_t)N * L.g.F * esz(L.dbl));
      const size_t solve_size = P->dbl ? 8 : 4;   // fp32 mode solves corrections in fp32 on every level
      const size_t scgs_bytes = d3 ? scgs3_smem_bytes(L.g.N, solve_size) : scgs_smem_bytes(N, solve_size);
      if (scgs_bytes + (d3 ? 1024 : 0) > (size_t)smem_optin)
        fail(STC_ERR_UNSUPPORTED, "too many timesteps for the shared-memory SCGS solve");

      P->lv.push_back(L);
    }
    const size_t F = g0.F, C = g0.C, ts = P->ts;
    P->rho = dalloc(P, (N + 1) * C * ts);
    P->rho_k = dalloc(P, (N + 1) * C * ts);
    P->rho_last = dalloc(P, (N + 1) * C * ts);
    P->mu = dalloc(P, N * C * ts);
    P->vstar = dalloc(P, N * F * ts);
    P->vcand = dalloc(P, N * F * ts);
    P->rho_c = dalloc(P, (N + 1) * C * ts);
    P->K_c = (int*)dalloc(P, N * sizeof(int));
    P->dguard = (double*)dalloc(P, 2 * P->lv.size() * sizeof(double));
    P->dlm = (double*)dalloc(P, sizeof(double));
    if (prm.lm_adapt) alloc_fieldset(P, P->xb, g0, P->dbl);
    if (prm.k_adapt) P->vprev = dalloc(P, (N + 1) * F * ts);
    P->lam = dalloc(P, N * F * ts);
    P->w = dalloc(P, N * F * ts);
    P->y = dalloc(P, N * F * ts);
    P->uk = dalloc(P, N * F * ts);
    P->gk = dalloc(P, (N + 1) * F * ts);
    P->dens = dalloc(P, (N + 1) * F * ts);
    P->powers = dalloc(P, (size_t)prm.taylor_kmax * C * ts);
    P->v0 = dalloc(P, F * ts);
    P->K = (int*)dalloc(P, N * sizeof(int));
    P->Kk = (int*)dalloc(P, N * sizeof(int));
    P->mterm = (double*)dalloc(P, (N + 1) * C * sizeof(double));
    P->mtmp0 = (double*)dalloc(P, C * sizeof(double));
    P->mtmp1 = (double*)dalloc(P, metric_tmp1_doubles(C, prm.metric_levels) * sizeof(double));
    P->dscal = (double*)dalloc(P, 16 * sizeof(double));
    P->derr = (int*)dalloc(P, sizeof(int));
    P->red = alloc_red(P, red_capacity(g0));
    P->ntrials = ao_trial_count(prm);
    if (P->ntrials > 1) {
      P->tv[0] = P->vcand;
      P->trho[0] = P->rho_c;
      P->tK[0] = P->K_c;
      P->ttmp0[0] = P->mtmp0;
      P->ttmp1[0] = P->mtmp1;
      for (int j = 0; j < P->ntrials; ++j) {
        if (j > 0) {
          P->tv[j] = dalloc(P, N * F * ts);
          P->trho[j] = dalloc(P, (N + 1) * C * ts);
          P->tK[j] = (int*)dalloc(P, N * sizeof(int));
          P->ttmp0[j] = (double*)dalloc(P, C * sizeof(double));
          P->ttmp1[j] = (double*)dalloc(P, metric_tmp1_doubles(C, prm.metric_levels) * sizeof(double));
        }
        P->tmterm[j] = (double*)dalloc(P, (N + 1) * C * sizeof(double));
        P->tred[j] = alloc_red(P, kReduceMaxBlocks);
        ck(cudaStreamCreateWithFlags(&P->tst[j], cudaStreamNonBlocking), "stream");
        ck(cudaEventCreateWithFlags(&P->tdone[j], cudaEventDisableTiming), "event");
      }
      P->terr = (int*)dalloc(P, kMaxTrials * sizeof(int));
      P->dtrial = (double*)dalloc(P, kMaxTrials * sizeof(double));
      ck(cudaEventCreateWithFlags(&P->tfork, cudaEventDisableTiming), "event");
      ck(cudaMallocHost(&P->htrial, kMaxTrials * (sizeof(double) + sizeof(int))), "pinned");
    }
    // projections run on at most N + 1 fields at once (stc_project on V or KKT_G)
    if (d3) {
      P->pscratch = dalloc(P, project3_scratch_elems(g0, N + 1) * ts);
      P->adv3 = dalloc(P, advect3_scratch_bytes(g0, ts));
      P->sc3 = dalloc(P, scgs3_thomas_scratch_bytes(g0, P->dbl ? 8 : 4));
      const Level& Lc = P->lv.back();
      P->lamb3_bytes = lamb3_scratch_bytes_max(g0, ts, Lc.g, esz(Lc.dbl));
      if (P->lamb3_bytes > 0) P->lamb3 = dalloc(P, P->lamb3_bytes);
    } else if (project_needs_scratch(g0, ts)) {
      P->pscratch = dalloc(P, (N + 1) * project_smem(g0, ts));
    }
    if (project_dct_fits(g0, ts)) {
      const size_t ne = project_dct_elems(g0);
      std::vector<double> tab(ne);
      project_dct_tables(g0, tab.data());
      P->dct = dalloc(P, ne * ts);
      // on the problem's stream, after dalloc's zeroing (a copy on another
      // stream could land before that memset)
      std::vector<float> tf(P->dbl ? 0 : ne);
      for (size_t e = 0; e < tf.size(); ++e) tf[e] = (float)tab[e];
      const void* src = P->dbl ? (const void*)tab.data() : (const void*)tf.data();
      ck(cudaMemcpyAsync(P->dct, src, ne * ts, cudaMemcpyHostToDevice, P->st), "h2d");
      ck(cudaStreamSynchronize(P->st), "sync");
    }
    ck(cudaMallocHost(&P->hscal, 16 * sizeof(double)), "pinned");
    ck(cudaMallocHost(&P->herr, sizeof(int)), "pinned");
    // inputs: rho_0 into rho[0] of every density buffer, v_0
    double mx = 0.0;
    for (size_t e = 0; e < C; ++e) mx = std::max(mx, std::fabs(rho0[e]));
    if (!(mx > 0.0)) fail(STC_ERR_INVALID_ARG, "rho0 must have a nonzero entry");
    P->rho_scale = mx;
    FieldRef r;
    r.count = C;
    r.dbl = P->dbl;
    r.ptr = P->rho;
    copy_in(P, r, rho0);
    r.ptr = P->rho_k;
    copy_in(P, r, rho0);
    r.ptr = P->rho_last;
    copy_in(P, r, rho0);
    r.ptr = P->rho_c;
    copy_in(P, r, rho0);
    for (int j = 1; j < P->ntrials; ++j) {
      r.ptr = P->trho[j];
      copy_in(P, r, rho0);
    }
    if (v0) {
      std::vector<double> vv(v0, v0 + F);
      // wall faces are not unknowns: keep them zero
      if (d3) {
        for (size_t f = 0; f < F; ++f) {
          int axis, k, j, i;
          if (f < (size_t)g0.Fx) {
            axis = 0;
            i = (int)(f % (g0.nx + 1));
            j = (int)((f / (g0.nx + 1)) % g0.ny);
            k = (int)(f / ((size_t)(g0.nx + 1) * g0.ny));
          } else if (f < (size_t)g0.Fxy) {
            axis = 1;
            const size_t q = f - g0.Fx;
            i = (int)(q % g0.nx);
            j = (int)((q / g0.nx) % (g0.ny + 1));
            k = (int)(q / ((size_t)g0.nx * (g0.ny + 1)));
          } else {
            axis = 2;
            const size_t q = f - g0.Fxy;
            i = (int)(q % g0.nx);
            j = (int)((q / g0.nx) % g0.ny);
            k = (int)(q / ((size_t)g0.nx * g0.ny));
          }
          const int p = axis == 0 ? i : (axis == 1 ? j : k);
          const int n = axis == 0 ? g0.nx : (axis == 1 ? g0.ny : g0.nz);
          if (p == n || (!g0.periodic && p == 0)) vv[f] = 0.0;   // walls / the unused periodic slot
        }
      } else {
        for (int j = 0; j < g0.ny; ++j) {
          vv[(size_t)j * (g0.nx + 1)] = 0.0;
          vv[(size_t)j * (g0.nx + 1) + g0.nx] = 0.0;
        }
        for (int i = 0; i < g0.nx; ++i) {
          vv[g0.Fx + i] = 0.0;
          vv[g0.Fx + (size_t)g0.ny * g0.nx + i] = 0.0;
        }
      }
      FieldRef rv;
      rv.count = F;
      rv.dbl = P->dbl;
      rv.ptr = P->v0;
      copy_in(P, rv, vv.data());
    }
    reset_state(P);
    ck(cudaStreamSynchronize(P->st), "sync");
  });
  if (s != STC_OK) {
    free_problem(P);
    return s;
  }
  *out = P;
  return STC_OK;
}

stc_status stc_destroy_problem(stc_problem* p) {
  if (!p) return STC_OK;
  if (p->st) cudaStreamSynchronize(p->st);
  else cudaDeviceSynchronize();
  free_problem(p);
  return STC_OK;
}

stc_status stc_set_keyframes(stc_problem* p, int count, const int* steps, const double* rho_star, const double* c) {
  if (!p || count < 0 || (count > 0 && (!steps || !rho_star))) {
    g_last_error = "invalid keyframe arguments";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    const Geom& g = p->lv[0].g;
    for (int k = 0; k < count; ++k)
      if (steps[k] < 1 || steps[k] > g.N) fail(STC_ERR_INVALID_ARG, "keyframe step outside 1..N");
    for (int a = 0; a < count; ++a)
      for (int b = a + 1; b < count; ++b)
        if (steps[a] == steps[b]) fail(STC_ERR_INVALID_ARG, "duplicate keyframe step");
    if (p->star) {
      cudaFree(p->star);
      for (auto& q : p->allocs)
        if (q == p->star) q = nullptr;
      p->star = nullptr;
      p->bytes -= p->star_bytes;
      p->star_bytes = 0;
    }
    p->key_steps.assign(steps, steps + count);
    p->key_c.assign(count, 1.0);
    if (c)
      for (int k = 0; k < count; ++k) p->key_c[k] = c[k];
    if (count > 0) {
      p->star_bytes = (size_t)count * g.C * sizeof(double);
      p->star = (double*)dalloc(p, p->star_bytes);
      ck(cudaMemcpyAsync(p->star, rho_star, (size_t)count * g.C * sizeof(double), cudaMemcpyHostToDevice, p->st),
         "h2d");
      ck(cudaStreamSynchronize(p->st), "sync");
    }
  });
}

stc_status stc_vcycle(stc_problem* p, int ncycles, double* nso_res_inf) {
  if (!p || ncycles < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    double f = 0.0;
    for (int c = 0; c < ncycles; ++c) f = run_vcycle(p, false, c == 0);
    if (ncycles == 0) {
      residual_norm(p, 0, 0, p->st);
      f = read_scalar(p, 0);
    }
    if (nso_res_inf) *nso_res_inf = f;
  });
}

stc_status stc_solve(stc_problem* p, double kkt_rel_tol, int max_admm, stc_report* report) {
  if (!p || max_admm < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  p->run = SolveRun{};
  p->run.rep.K_final = p->prm.K;
  stc_status s = guarded(p, [&]() {
    solve_begin(p, kkt_rel_tol, max_admm);
    while (p->run.phase != 2) {
      solve_head(p);
      while (solve_wants_cycle(p)) solve_cycle_done(p, run_vcycle(p, p->prm.lm_adapt != 0));
      solve_tail(p);
    }
  });
  if (report) *report = p->run.rep;
  if (s != STC_OK) return s;
  if (!p->run.converged) {
    g_last_error = "ADMM iteration cap reached";
    return STC_ERR_NOT_CONVERGED;
  }
  return STC_OK;
}

// ---- resumable solve and batched NSO cycles --------------------------------

stc_status stc_solve_begin(stc_problem* p, double kkt_rel_tol, int max_admm) {
  if (!p || max_admm < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  p->run = SolveRun{};
  return guarded(p, [&]() { solve_begin(p, kkt_rel_tol, max_admm); });
}

stc_status stc_solve_phase(const stc_problem* p, int* phase, int* wants_cycle) {
  if (!p || !phase) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  *phase = p->run.phase;
  if (wants_cycle) *wants_cycle = solve_wants_cycle(p) ? 1 : 0;
  return STC_OK;
}

stc_status stc_solve_head(stc_problem* p) {
  if (!p || p->run.phase != 0) {
    g_last_error = "stc_solve_head: no ADMM iteration is due";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() { solve_head(p); });
}

stc_status stc_solve_tail(stc_problem* p) {
  if (!p || p->run.phase != 1 || solve_wants_cycle(p)) {
    g_last_error = "stc_solve_tail: the NSO solve of this iteration is not finished";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() { solve_tail(p); });
}

stc_status stc_solve_report(const stc_problem* p, stc_report* report, int* converged) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  if (report) *report = p->run.rep;
  if (converged) *converged = p->run.converged ? 1 : 0;
  return STC_OK;
}

}  // extern "C"

struct stc_batch {
  cudaStream_t st = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<std::pair<const stc_problem*, long long>> key;   // composition of exec
  long long launches = 0;
};

extern "C" {

stc_status stc_batch_create(void* cuda_stream, stc_batch** out) {
  if (!out) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  *out = new (std::nothrow) stc_batch();
  if (!*out) {
    g_last_error = "host allocation failed";
    return STC_ERR_OOM;
  }
  (*out)->st = (cudaStream_t)cuda_stream;
  return STC_OK;
}

stc_status stc_batch_destroy(stc_batch* b) {
  if (!b) return STC_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
  return STC_OK;
}

stc_status stc_batch_nso_cycle(stc_batch* b, stc_problem* const* probs, int n, int* cycled, stc_status* status) {
  if (!b || n < 0 || (n > 0 && !probs)) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  std::vector<stc_problem*> go;
  for (int k = 0; k < n; ++k) {
    if (status) status[k] = STC_OK;
    stc_problem* p = probs[k];
    if (!p || p->broken || !solve_wants_cycle(p)) continue;
    const stc_status sk = guarded(p, [&]() {
      ensure_vgraph(p, false);
      ck(cudaStreamSynchronize(p->st), "sync");   // the problem's own work before the batched launch
    });
    if (sk != STC_OK) {
      if (status) status[k] = sk;
      continue;
    }
    go.push_back(p);
  }
  if (cycled) *cycled = (int)go.size();
  if (go.empty()) return STC_OK;
  std::vector<std::pair<const stc_problem*, long long>> key;
  for (stc_problem* p : go) key.emplace_back(p, p->vgraph_version);
  try {
    if (!b->exec || key != b->key) {
      if (b->exec) {
        ck(cudaGraphExecDestroy(b->exec), "graph destroy");
        b->exec = nullptr;
      }
      cudaGraph_t root = nullptr;
      ck(cudaGraphCreate(&root, 0), "graph create");
      cudaError_t e = cudaSuccess;
      for (stc_problem* p : go) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, root, nullptr, 0, p->vgraph_src);
        if (e != cudaSuccess) break;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, root, 0);
      cudaGraphDestroy(root);
      ck(e, "batched graph");
      b->key = key;
    }
    ck(cudaGraphLaunch(b->exec, b->st), "batched graph launch");
    ck(cudaStreamSynchronize(b->st), "sync");
  } catch (const StcError& e) {
    g_last_error = e.msg;
    return e.code;
  }
  // each problem's norm, then its LM decision (Sec. 5)
  for (int k = 0; k < n; ++k) {
    stc_problem* p = probs[k];
    if (std::find(go.begin(), go.end(), p) == go.end()) continue;
    const stc_status sk = guarded(p, [&]() {
      p->launches += p->graph_launches;
      solve_cycle_done(p, read_scalar(p, 0, false, p->prm.lm_adapt != 0));
    });
    if (status) status[k] = sk;
  }
  return STC_OK;
}

stc_status stc_solve_history(const stc_problem* p, double* out, size_t len, int* count) {
  if (!p || (!out && len > 0)) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  const size_t n = p->solve_hist.size() / 3;
  for (size_t k = 0; k < 3 * n && k < len; ++k) out[k] = p->solve_hist[k];
  if (count) *count = (int)n;
  return STC_OK;
}

stc_status stc_get_forces(const stc_problem* p, double* u, size_t len) {
  return stc_get_field(p, STC_FIELD_U, 0, u, len);
}
stc_status stc_get_density(const stc_problem* p, double* rho, size_t len) {
  return stc_get_field(p, STC_FIELD_RHO, 0, rho, len);
}
stc_status stc_get_velocity(const stc_problem* p, double* v, size_t len) {
  return stc_get_field(p, STC_FIELD_V, 0, v, len);
}

stc_status stc_get_field(const stc_problem* cp, int field, int level, double* out, size_t len) {
  stc_problem* p = const_cast<stc_problem*>(cp);
  if (!p || !out) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    FieldRef r = field_ref(p, field, level);
    if (len != r.count) fail(STC_ERR_INVALID_ARG, "length does not match the field size");
    copy_out(p, r, out);
  });
}

stc_status stc_set_field(stc_problem* p, int field, int level, const double* in, size_t len) {
  if (!p || !in) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    FieldRef r = field_ref(p, field, level);
    if (len != r.count) fail(STC_ERR_INVALID_ARG, "length does not match the field size");
    copy_in(p, r, in);
    if (field == STC_FIELD_VSTAR || field == STC_FIELD_RHO) p->rho_at_vstar = false;
  });
}

stc_status stc_level_info(const stc_problem* p, int* nlevels, int level, int* nx, int* ny) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  if (nlevels) *nlevels = (int)p->lv.size();
  if (level < 0 || level >= (int)p->lv.size()) {
    g_last_error = "level out of range";
    return STC_ERR_INVALID_ARG;
  }
  if (nx) *nx = p->lv[level].g.nx;
  if (ny) *ny = p->lv[level].g.ny;
  return STC_OK;
}

stc_status stc_level_dims(const stc_problem* p, int level, int* nx, int* ny, int* nz) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  if (level < 0 || level >= (int)p->lv.size()) {
    g_last_error = "level out of range";
    return STC_ERR_INVALID_ARG;
  }
  const Geom& g = p->lv[level].g;
  if (nx) *nx = g.nx;
  if (ny) *ny = g.ny;
  if (nz) *nz = g.dim == 3 ? g.nz : 0;
  return STC_OK;
}

stc_status stc_simulate(stc_problem* p, double picard_tol, int max_iter, int* iters) {
  if (!p || !(picard_tol > 0) || max_iter < 1) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    sim_alloc(p);
    const Geom& g = p->lv[0].g;
    int total = 0;
    for (int t = 0; t < g.N; ++t) total += picard_step(p, t, picard_tol, max_iter);
    forward(p, p->lv[0].x.v, p->rho, p->K, p->st);
    p->rho_at_vstar = false;
    (void)read_scalar(p, 0);   // surfaces the sweep's device error flags
    if (iters) *iters = total;
  });
}

stc_status stc_simulate_adjoint(stc_problem* p, double picard_tol, int max_iter, int with_step0, int* iters) {
  if (!p || !(picard_tol > 0) || max_iter < 1 || with_step0 < 0 || with_step0 > 1) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    sim_alloc(p);
    const Geom& g = p->lv[0].g;
    const size_t N = g.N, fb = (size_t)g.F * p->ts;
    // density adjoint: the sweep's metric terms are -dL/drho
    launch_sim_copy<double, double>((N + 1) * g.C, p->sim_grho, -1.0, p->mterm, p->st);
    ck(cudaMemsetAsync(p->dens, 0, (N + 1) * fb, p->st), "memset");
    if (with_step0) ck(cudaMemsetAsync(p->sim_l0, 0, (size_t)g.C * p->ts, p->st), "memset");
    adjoint(p, p->lv[0].x.v, p->rho, p->K, nullptr, 0.0, 1.0, p->dens, p->st, with_step0 ? 0 : 1,
            with_step0 ? p->sim_l0 : nullptr);
    if (!with_step0) ck(cudaMemsetAsync(p->sim_l0, 0, (size_t)g.C * p->ts, p->st), "memset");   // not formed
    // velocity adjoint, i = N-1 .. 0: xi = Pi_i^T a = dt z, a <- dens_i + z
    ck(cudaMemcpyAsync(p->sim_a0, p->sim_aN, fb, cudaMemcpyDeviceToDevice, p->st), "copy");
    int total = 0;
    for (int i = (int)N - 1; i >= 0; --i) {
      total += picard_adjoint_step(p, i, p->sim_a0, picard_tol, max_iter);
      dispatch(p->dbl, [&](auto tag) {
        using T = decltype(tag);
        launch_sim_axpby<T>((size_t)g.F, g.dt, (const T*)p->sim_w2, 0.0, nullptr,
                            (T*)((char*)p->sim_gu + i * fb), p->st);
        launch_sim_axpby<T>((size_t)g.F, 1.0, (const T*)((char*)p->dens + i * fb), 1.0, (const T*)p->sim_w2,
                            (T*)p->sim_a0, p->st);
      });
      count(p, 2);
    }
    (void)read_scalar(p, 0);
    if (iters) *iters = total;
  });
}

stc_status stc_copy_field_device(stc_problem* p, int field, int level, void* buffer, size_t len, int buffer_is_double,
                                 int to_field, double scale) {
  if (!p || !buffer || buffer_is_double < 0 || buffer_is_double > 1 || to_field < 0 || to_field > 1) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    FieldRef r = field_ref(p, field, level);
    if (len != r.count) fail(STC_ERR_INVALID_ARG, "length does not match the field size");
    const bool fdbl = r.kind == 1 || r.dbl;
    auto go = [&](auto ftag, auto btag) {
      using Tf = decltype(ftag);
      using Tb = decltype(btag);
      if (to_field) launch_sim_copy<Tb, Tf>(len, (const Tb*)buffer, scale, (Tf*)r.ptr, p->st);
      else launch_sim_copy<Tf, Tb>(len, (const Tf*)r.ptr, scale, (Tb*)buffer, p->st);
    };
    if (fdbl && buffer_is_double) go(double(), double());
    else if (fdbl) go(double(), float());
    else if (buffer_is_double) go(float(), double());
    else go(float(), float());
    count(p, 1);
    check_launch("copy");
    if (to_field && (field == STC_FIELD_VSTAR || field == STC_FIELD_RHO)) p->rho_at_vstar = false;
  });
}

stc_status stc_level_steps(const stc_problem* p, int level, int* num_steps, double* dt) {
  if (!p || level < 0 || level >= (int)p->lv.size()) {
    g_last_error = "level out of range";
    return STC_ERR_INVALID_ARG;
  }
  if (num_steps) *num_steps = p->lv[level].g.N;
  if (dt) *dt = p->lv[level].g.dt;
  return STC_OK;
}

stc_status stc_advect(stc_problem* p, int source_field) {
  if (!p || (source_field != STC_FIELD_VSTAR && source_field != STC_FIELD_V)) {
    g_last_error = "source must be STC_FIELD_VSTAR or STC_FIELD_V";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    const void* vel = source_field == STC_FIELD_V ? p->lv[0].x.v : p->vstar;
    forward(p, vel, p->rho, p->K, p->st);
    p->rho_at_vstar = source_field == STC_FIELD_VSTAR;
    read_scalar(p, 0);   // synchronise and surface device errors
  });
}

stc_status stc_get_taylor_orders(const stc_problem* p, int* K, size_t len) {
  if (!p || !K || len != (size_t)p->lv[0].g.N) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  stc_problem* q = const_cast<stc_problem*>(p);
  return guarded(q, [&]() {
    ck(cudaMemcpyAsync(K, q->K, len * sizeof(int), cudaMemcpyDeviceToHost, q->st), "d2h");
    ck(cudaStreamSynchronize(q->st), "sync");
  });
}

stc_status stc_metric_terms(stc_problem* p) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    metric_terms(p, p->rho, p->st);
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_adjoint(stc_problem* p, int source_field, double alpha, double beta) {
  if (!p || (source_field != STC_FIELD_VSTAR && source_field != STC_FIELD_V)) {
    g_last_error = "source must be STC_FIELD_VSTAR or STC_FIELD_V";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    const void* vel = source_field == STC_FIELD_V ? p->lv[0].x.v : p->vstar;
    adjoint(p, vel, p->rho, p->K, p->w, alpha, beta, p->y, p->st);
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_project(stc_problem* p, int field, int first, int count) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    if (field != STC_FIELD_V && field != STC_FIELD_U && field != STC_FIELD_VSTAR && field != STC_FIELD_Y &&
        field != STC_FIELD_W && field != STC_FIELD_KKT_U && field != STC_FIELD_KKT_G && field != STC_FIELD_Z)
      fail(STC_ERR_INVALID_ARG, "not a face field");
    FieldRef r = field_ref(p, field, 0);
    const Geom& g = p->lv[0].g;
    const size_t slabs = r.count / g.F;
    if (first < 0 || count < 0 || (size_t)first + (size_t)count > slabs)
      fail(STC_ERR_INVALID_ARG, "slab range outside the field");
    project(p, (char*)r.ptr + (size_t)first * g.F * p->ts, count, p->st);
    if (field == STC_FIELD_VSTAR) p->rho_at_vstar = false;
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_ao(stc_problem* p, int iters, int warm_start) {
  if (!p || iters < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    ao(p, iters, warm_start != 0, p->st);
    read_scalar(p, 0);
  });
}

stc_status stc_ao_trace(const stc_problem* p, int* halvings, size_t len, int* count) {
  if (!p || (!halvings && len > 0)) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  const size_t n = p->ao_trace.size();
  for (size_t k = 0; k < n && k < len; ++k) halvings[k] = p->ao_trace[k];
  if (count) *count = (int)n;
  return STC_OK;
}

stc_status stc_prepare_targets(stc_problem* p) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    prepare_targets(p, p->st);
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_nso_residual(stc_problem* p, int level, double* inf) {
  if (!p || level < 0 || level >= (int)p->lv.size()) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    residual_norm(p, level, 3, p->st);
    const double v = read_scalar(p, 3);
    if (inf) *inf = v;
  });
}

stc_status stc_nso_solve(stc_problem* p, double f_target, int max_cycles, int* cycles, double* f_inf) {
  if (!p || max_cycles < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    nso_begin(p);
    residual_norm(p, 0, 0, p->st);
    double f = read_scalar(p, 0);
    int c = 0;
    bool give_up = false;
    while ((c < 1 || f > f_target) && c < max_cycles && !give_up) {
      f = nso_cycle(p, f, &give_up);
      ++c;
    }
    if (cycles) *cycles = c;
    if (f_inf) *f_inf = f;
  });
}

stc_status stc_lm_info(const stc_problem* p, double* lm_shift, int* rejected) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  if (lm_shift) *lm_shift = p->lm;
  if (rejected) *rejected = p->rejected;
  return STC_OK;
}

stc_status stc_smooth(stc_problem* p, int level, int sweeps) {
  if (!p || level < 0 || level >= (int)p->lv.size() || sweeps < 0) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    smooth(p, level, sweeps, p->st);
    check_launch("smooth");
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_restrict(stc_problem* p, int level) {
  if (!p || level < 0 || level + 1 >= (int)p->lv.size()) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    restrict_level(p, level, p->st);
    check_launch("restrict");
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_prolong_correct(stc_problem* p, int level) {
  if (!p || level < 0 || level + 1 >= (int)p->lv.size()) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    prolong_level(p, level, p->st);
    check_launch("prolong");
    ck(cudaStreamSynchronize(p->st), "sync");
  });
}

stc_status stc_kkt_residual(stc_problem* p, double* norm) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    kkt(p, p->st);
    const double v = read_scalar(p, 1);
    if (norm) *norm = std::sqrt(v);
  });
}

stc_status stc_admm_update(stc_problem* p, double* drho) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    admm_update(p, p->st);
    const double v = read_scalar(p, 2);
    if (drho) *drho = v;
  });
}

stc_status stc_set_penalty(stc_problem* p, double K, double beta) {
  if (!p || !(K > 0) || !(beta > 0) || !std::isfinite(K) || !std::isfinite(beta)) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() { set_penalty_impl(p, K, beta); });
}

stc_status stc_launch_count(const stc_problem* p, long long* launches) {
  if (!p || !launches) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  *launches = p->launches;
  return STC_OK;
}

stc_status stc_set_kernel_timing(stc_problem* p, int enable) {
  if (!p) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  return guarded(p, [&]() {
    drop_vgraphs(p);
    p->timing = enable != 0;
    // one event pair per finest-level colour launch of a cycle (the finest
    // level is smoothed with events only when it is not the coarsest)
    const size_t need = p->lv.size() > 1 ? (size_t)(1 << p->lv[0].g.dim) * (p->prm.pre + p->prm.post) : 0;
    for (int kind = 0; kind < 2; ++kind) {
      p->timed_ms[kind] = 0.0;
      p->timed_launches[kind] = 0;
      while (p->timing && p->ev_start[kind].size() < need) {
        cudaEvent_t a, b;
        ck(cudaEventCreate(&a), "event");
        ck(cudaEventCreate(&b), "event");
        p->ev_start[kind].push_back(a);
        p->ev_stop[kind].push_back(b);
      }
    }
  });
}

stc_status stc_kernel_timing(const stc_problem* p, double* total_ms, long long* launches) {
  return stc_kernel_timing_of(p, 0, total_ms, launches);
}

stc_status stc_kernel_timing_of(const stc_problem* p, int kind, double* total_ms, long long* launches) {
  if (!p || kind < 0 || kind > 1) {
    g_last_error = "invalid argument";
    return STC_ERR_INVALID_ARG;
  }
  if (total_ms) *total_ms = p->timed_ms[kind];
  if (launches) *launches = p->timed_launches[kind];
  return STC_OK;
}

stc_status stc_dct_tables(int nx, int ny, double* out, size_t len) {
  if (nx < 1 || ny < 1 || !out) {
    stc::set_last_error("invalid argument");
    return STC_ERR_INVALID_ARG;
  }
  Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.dim = 2;
  g.nz = 1;
  g.h = 1.0 / nx;
  if (len < project_dct_elems(g)) {
    stc::set_last_error("output shorter than 2 nx^2 + 2 ny^2 + nx ny");
    return STC_ERR_INVALID_ARG;
  }
  project_dct_tables(g, out);
  return STC_OK;
}

stc_status stc_problem_bytes(const stc_params* params, int nkeys, size_t* bytes) {
  if (!params || !bytes || nkeys < 0 || !params_valid(*params)) {
    stc::set_last_error("invalid parameters");
    return STC_ERR_INVALID_ARG;
  }
  *bytes = plan_bytes(*params, nkeys);
  return STC_OK;
}

stc_status stc_memory_bytes(const stc_problem* p, size_t* bytes) {
  if (!p || !bytes) {
    g_last_error = "null argument";
    return STC_ERR_INVALID_ARG;
  }
  *bytes = p->bytes;
  return STC_OK;
}

}  // extern "C"
