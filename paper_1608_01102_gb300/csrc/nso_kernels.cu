// NSO subproblem kernels: residual f of Eq. KKTAO, the temporally augmented
// SCGS smoother of Sec. 4.3 / Eq. HESS, the STFAS transfer operators R and P
// (Sec. 4.3, Alg. 2) and reductions.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include "stc_internal.cuh"
#include "stc_kernels.h"

namespace stc {

// ---------------------------------------------------------------------------
// f(v, pbar, u, p)  (Eq. KKTAO with v_0 fixed, z = v* - lambda/K):
//   row 1, faces, t = 1..N : a(v_t - z_t)[t<N] - u_t/dt [t<N] + u_{t-1}/dt
//                            + (dAdv(v_t))^T u_{t-1} + grad pbar_t
//   row 2, cells, t = 1..N : -div v_t
//   row 3, faces, t = 0..N-1: (v_{t+1} - v_t)/dt + Adv(v_{t+1}) - u_t + grad p_{t+1}
//   row 4, cells, t = 0..N-1: -div u_t
// out = sf * f + sr * res (res may be null).  Rows dropped by the fixed v_0
// (row 1/2 at t = 0) and wall-face rows are written as 0.
// Thread x: element index e (a face if e < F, and a cell if e < C);
// blockIdx.y: time t in [0, N].  The rows are evaluated by the helpers below,
// which the SCGS kernel also calls for its own cells (same arithmetic).
// ---------------------------------------------------------------------------
// row 1 at interior face e = (j, i) of direction isx, time t >= 1
template <class T>
__device__ __forceinline__ T nso_row1(const Geom& g, const CState<T>& x, const T* __restrict__ z, int t, int e,
                                      bool isx, int j, int i) {
  const T* vt = x.v + (size_t)t * g.F;
  const T* um = x.u + (size_t)(t - 1) * g.F;
  const T* pb = x.pbar + (size_t)t * g.C;
  T val = ld(um + e) * pick<T>(g.idt, g.idtf);
  if (g.self_adv) val += T(g.self_adv) * (isx ? jtu_x(g, vt, um, j, i) : jtu_y(g, vt, um, j, i));
  val += isx ? grad_x(g, pb, j, i) : grad_y(g, pb, j, i);
  if (t < g.N) {
    const T* ut = x.u + (size_t)t * g.F;
    val += pick<T>(g.a, g.af) * (ld(vt + e) - ld(z + (size_t)t * g.F + e)) - ld(ut + e) * pick<T>(g.idt, g.idtf);
  }
  return val;
}
// row 3 at interior face e = (j, i), time t <= N - 1
template <class T>
__device__ __forceinline__ T nso_row3(const Geom& g, const CState<T>& x, int t, int e, bool isx, int j, int i) {
  const T* vn = x.v + (size_t)(t + 1) * g.F;
  const T* vt = x.v + (size_t)t * g.F;
  const T* pp = x.p + (size_t)t * g.C;
  T val = (ld(vn + e) - ld(vt + e)) * pick<T>(g.idt, g.idtf) - ld(x.u + (size_t)t * g.F + e);
  if (g.self_adv) val += T(g.self_adv) * (isx ? adv_x(g, vn, j, i) : adv_y(g, vn, j, i));
  val += isx ? grad_x(g, pp, j, i) : grad_y(g, pp, j, i);
  return val;
}

template <class T>
__global__ void nso_residual_kernel(Geom g, CState<T> x, const T* __restrict__ z,
                                   CState<T> res, State<T> out, T sf, T sr, double* sq, RedScratch rs,
                                   const double* only_if_undone) {
  pdl_wait();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (t > g.N) return;
  // conditional form (after a guarded coarse-grid correction): the residual
  // already in `out` is current unless the correction was undone
  if (only_if_undone && only_if_undone[1] <= only_if_undone[0]) return;
  T acc = T(0);   // sum of squares of this thread's (at most 4) outputs; fp64 across threads
  const int N = g.N;
  const T idt = pick<T>(g.idt, g.idtf);
  const T sa = T(g.self_adv);
  if (e < g.F) {
    int j, i;
    bool isx = e < g.Fx;
    if (isx) {
      j = e / (g.nx + 1);
      i = e - j * (g.nx + 1);
    } else {
      int q = e - g.Fx;
      j = q / g.nx;
      i = q - j * g.nx;
    }
    bool interior = isx ? xf_interior(g, j, i) : yf_interior(g, j, i);
    // row 1 at time t (t >= 1)
    if (t >= 1) {
      T val = T(0);
      if (interior) {
        val = nso_row1(g, x, z, t, e, isx, j, i) * sf;
        if (res.v) val += sr * ld(res.v + (size_t)t * g.F + e);
      }
      out.v[(size_t)t * g.F + e] = val;
      acc += val * val;
    } else {
      out.v[e] = T(0);
    }
    // row 3 at time t (t < N)
    if (t < N) {
      T val = T(0);
      if (interior) {
        val = nso_row3(g, x, t, e, isx, j, i) * sf;
        if (res.u) val += sr * ld(res.u + (size_t)t * g.F + e);
      }
      out.u[(size_t)t * g.F + e] = val;
      acc += val * val;
    }
  }
  if (e < g.C) {
    const int j = e / g.nx, i = e - (e / g.nx) * g.nx;
    if (t >= 1) {
      T val = -divergence(g, x.v + (size_t)t * g.F, j, i) * sf;
      if (res.pbar) val += sr * ld(res.pbar + (size_t)t * g.C + e);
      out.pbar[(size_t)t * g.C + e] = val;
      acc += val * val;
    } else {
      out.pbar[e] = T(0);
    }
    if (t < N) {
      T val = -divergence(g, x.u + (size_t)t * g.F, j, i) * sf;
      if (res.p) val += sr * ld(res.p + (size_t)t * g.C + e);
      out.p[(size_t)t * g.C + e] = val;
      acc += val * val;
    }
  }
  if (sq) block_sum_ordered((double)acc, sq, rs);
}

// ---------------------------------------------------------------------------
// f - res restricted to what the SCGS sweep of one colour reads: the rows at
// the faces of that colour's cells (x-faces of rows j = py mod 2, y-faces of
// columns i = px mod 2) and at its cells; other entries of `out` are left as
// they are.  Same rows and arithmetic as nso_residual_kernel with sf = 1,
// sr = -1.  Thread x: index over (x-faces, y-faces, cells) of the colour;
// blockIdx.y: time t in [0, N].
// ---------------------------------------------------------------------------
template <class T>
__global__ void nso_residual_colour_kernel(Geom g, CState<T> x, const T* __restrict__ z, CState<T> res,
                                           State<T> out, int px, int py, const double* only_if_undone) {
  pdl_wait();
  const int t = blockIdx.y;
  if (t > g.N) return;
  if (only_if_undone && only_if_undone[1] <= only_if_undone[0]) return;
  const int N = g.N;
  const int nrx = (g.ny - py + 1) / 2;          // x-face rows j = py, py + 2, ...
  const int ncy = (g.nx - px + 1) / 2;          // y-face columns i = px, px + 2, ...
  const int nxf = nrx * (g.nx + 1), nyf = (g.ny + 1) * ncy;
  const int ncells = ((g.nx - px + 1) / 2) * nrx;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nxf + nyf) {
    int j, i, f;
    bool isx = e < nxf;
    if (isx) {
      const int r = e / (g.nx + 1);
      i = e - r * (g.nx + 1);
      j = py + 2 * r;
      f = xf(g, j, i);
    } else {
      const int q = e - nxf;
      const int r = q / ncy;
      j = r;
      i = px + 2 * (q - r * ncy);
      f = yf(g, j, i);
    }
    const bool interior = isx ? xf_interior(g, j, i) : yf_interior(g, j, i);
    if (t >= 1) {
      T val = T(0);
      if (interior) {
        val = nso_row1(g, x, z, t, f, isx, j, i);
        if (res.v) val -= ld(res.v + (size_t)t * g.F + f);
      }
      out.v[(size_t)t * g.F + f] = val;
    }
    if (t < N) {
      T val = T(0);
      if (interior) {
        val = nso_row3(g, x, t, f, isx, j, i);
        if (res.u) val -= ld(res.u + (size_t)t * g.F + f);
      }
      out.u[(size_t)t * g.F + f] = val;
    }
    return;
  }
  e -= nxf + nyf;
  if (e < ncells) {
    const int ncx = (g.nx - px + 1) / 2;
    const int j = py + 2 * (e / ncx), i = px + 2 * (e % ncx);
    const int c = cidx(g, j, i);
    if (t >= 1) {
      T val = -divergence(g, x.v + (size_t)t * g.F, j, i);
      if (res.pbar) val -= ld(res.pbar + (size_t)t * g.C + c);
      out.pbar[(size_t)t * g.C + c] = val;
    }
    if (t < N) {
      T val = -divergence(g, x.u + (size_t)t * g.F, j, i);
      if (res.p) val -= ld(res.p + (size_t)t * g.C + c);
      out.p[(size_t)t * g.C + c] = val;
    }
  }
}

// ---------------------------------------------------------------------------
// SCGS: one colour.  For a cell (j,i) the local unknowns per time block are
// B_u(t) = {u_t on the 4 faces, p_{t+1}} and B_v(t) = {v_t on the faces,
// pbar_t}, ordered B_u(0), B_v(1), B_u(1), ..., B_u(N-1), B_v(N).  The local
// Jacobian is the Eq. HESS restriction: diagonal blocks [[aI, g],[g^T, 0]] and
// [[-I, g],[g^T, 0]]; couplings -I/dt (v_t with u_t) and I/dt + dAdv_loc(v_{t+1})
// (u_t with v_{t+1}) and its transpose; the v diagonal carries the
// Levenberg-Marquardt shift.  It is solved by block Thomas elimination.  Every
// modified diagonal block keeps the saddle form [[A4, g],[g^T, 0]] with A4
// symmetric definite, which is solved by LDL^T plus a Schur step on g.
// rhs = -(f - res), read from a residual buffer computed for this colour.
// ---------------------------------------------------------------------------

// d Adv_f / d v_g for f, g in (L, R, B, T) faces of cell (j,i), at field v.
// (T: element type of v; R: arithmetic type of J)
template <class T, class R = T>
__device__ void local_adv_jac(const Geom& g, const T* v, int j, int i, R J[4][4]) {
  const R ih = pick<R>(g.ih, g.ihf);
  // node interior flags at the four corners
  auto an = [&](int jj, int ii) -> R {
    return (ii > 0 && ii < g.nx && jj > 0 && jj < g.ny) ? R(1) : R(0);
  };
  const R a00 = an(j, i), a10 = an(j + 1, i), a01 = an(j, i + 1), a11 = an(j + 1, i + 1);
  const R w00 = node_omega<T, R>(g, v, j, i), w10 = node_omega<T, R>(g, v, j + 1, i);
  const R w01 = node_omega<T, R>(g, v, j, i + 1), w11 = node_omega<T, R>(g, v, j + 1, i + 1);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) J[r][c] = R(0);
  // f = L (x-face (j,i)), s = -1
  if (xf_interior(g, j, i)) {
    R wb = R(0.5) * (w00 + w10), tv = tv_x<T, R>(g, v, j, i);
    // d wbar / d(L,R,B,T)
    R dL = R(0.5) * (-a00 + a10) * ih, dB = R(0.5) * a00 * ih, dT = R(0.5) * a10 * ih;
    J[0][0] = -(dL * tv);
    J[0][2] = -(dB * tv + wb * R(0.25));
    J[0][3] = -(dT * tv + wb * R(0.25));
  }
  // f = R (x-face (j,i+1)), s = -1
  if (xf_interior(g, j, i + 1)) {
    R wb = R(0.5) * (w01 + w11), tv = tv_x<T, R>(g, v, j, i + 1);
    R dR = R(0.5) * (-a01 + a11) * ih, dB = -R(0.5) * a01 * ih, dT = -R(0.5) * a11 * ih;
    J[1][1] = -(dR * tv);
    J[1][2] = -(dB * tv + wb * R(0.25));
    J[1][3] = -(dT * tv + wb * R(0.25));
  }
  // f = B (y-face (j,i)), s = +1
  if (yf_interior(g, j, i)) {
    R wb = R(0.5) * (w00 + w01), tv = tv_y<T, R>(g, v, j, i);
    R dB = R(0.5) * (a00 - a01) * ih, dL = -R(0.5) * a00 * ih, dR = -R(0.5) * a01 * ih;
    J[2][2] = dB * tv;
    J[2][0] = dL * tv + wb * R(0.25);
    J[2][1] = dR * tv + wb * R(0.25);
  }
  // f = T (y-face (j+1,i)), s = +1
  if (yf_interior(g, j + 1, i)) {
    R wb = R(0.5) * (w10 + w11), tv = tv_y<T, R>(g, v, j + 1, i);
    R dT = R(0.5) * (a10 - a11) * ih, dL = R(0.5) * a10 * ih, dR = R(0.5) * a11 * ih;
    J[3][3] = dT * tv;
    J[3][0] = dL * tv + wb * R(0.25);
    J[3][1] = dR * tv + wb * R(0.25);
  }
}

// Solve [[A, g], [g^T, 0]] [X; y] = [B; q] for NC right-hand sides.  A is the
// 4x4 symmetric face block, definite (either sign): LDL^T without pivoting,
// solves for the NC columns and for g, then the Schur step on g.  On return B
// holds X and Y holds y.
template <class T, int NC>
__device__ __forceinline__ void saddle_solve(T A[4][4], const T gv[4], T B[4][NC], const T q[NC], T Y[NC]) {
  T dinv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T d = A[k][k];
#pragma unroll
    for (int s = 0; s < k; ++s) d -= A[k][s] * A[k][s] * A[s][s];
    A[k][k] = d;
    const T id = T(1) / d;
    dinv[k] = id;
#pragma unroll
    for (int r = k + 1; r < 4; ++r) {
      T l = A[r][k];
#pragma unroll
      for (int s = 0; s < k; ++s) l -= A[r][s] * A[k][s] * A[s][s];
      A[r][k] = l * id;
    }
  }
  T X[4][NC + 1];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
#pragma unroll
    for (int c = 0; c < NC; ++c) X[r][c] = B[r][c];
    X[r][NC] = gv[r];
  }
#pragma unroll
  for (int c = 0; c <= NC; ++c) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T s = X[r][c];
#pragma unroll
      for (int k = 0; k < r; ++k) s -= A[r][k] * X[k][c];
      X[r][c] = s;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) X[r][c] *= dinv[r];
#pragma unroll
    for (int r = 3; r >= 0; --r) {
      T s = X[r][c];
#pragma unroll
      for (int k = r + 1; k < 4; ++k) s -= A[k][r] * X[k][c];
      X[r][c] = s;
    }
  }
  T sgg = T(0);
#pragma unroll
  for (int r = 0; r < 4; ++r) sgg += gv[r] * X[r][NC];
  const T isgg = T(1) / sgg;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T sgb = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) sgb += gv[r] * X[r][c];
    const T y = (sgb - q[c]) * isgg;
    Y[c] = y;
#pragma unroll
    for (int r = 0; r < 4; ++r) B[r][c] = X[r][c] - X[r][NC] * y;
  }
}

// One CTA smooths `cpb` cells of one colour.  Block order of a cell's time
// column: B_u(0), B_v(1), B_u(1), ..., B_u(N-1), B_v(N).  Every u block
// D_u = [[-I, g], [g^T, 0]] has the closed-form inverse
//   [[-P, gh], [gh^T, 1/|g|^2]],  P = I - g g^T / |g|^2,  gh = g / |g|^2
// (on the cell's active faces), so all u blocks are eliminated at once,
// leaving a symmetric block-tridiagonal system over the N v blocks:
//   S_t  = (a_t + lm) I + [t<N] P / dt^2 + U_{t-1}^T P U_{t-1}     (v_t pivot face block)
//   O_t  = -P U_t / dt                                            (v_t -> v_{t+1} coupling)
//   R_t  = b_v(t) + [t<N] y_t / dt - U_{t-1}^T y_{t-1}            (faces; y = D_u^{-1} b_u)
// with U_t = I/dt + dAdv_loc(v_{t+1}).  That system is solved by cyclic
// reduction: at stride s the blocks j = s, 3s, 5s, ... are eliminated in
// parallel (each a saddle solve with 9 right-hand sides: its left and right
// couplings and its right-hand side), then the blocks j = 0, 2s, 4s, ...
// gather both neighbours' contributions; after log2(N) levels block 0 is
// solved and the levels are unwound.  Each saddle pivot is solved after an
// exact gamma g g^T shift of its face block (x unchanged, multiplier shifted
// by gamma q) that keeps the block definite.  Phases:
//  A (parallel over cells x timesteps): U_t, b_u(t), b_v(t+1) into shared memory;
//  A2 (parallel): y_t; the v blocks' S, R and couplings;
//  B (one warp per cell, one lane per block): the cyclic reduction;
//  C (parallel): u_t = y_t + D_u^{-1} [v_t/dt - U_t v_{t+1}; 0]; x += omega delta.
// State type T and solve type S: the fp32 mode's fp64 coarsest level solves in fp32.
constexpr int kCrStride = 77;   // per-block record, odd so a warp's lanes hit distinct banks
enum : int { CR_A = 0, CR_R = 10, CR_C = 15, CR_ZL = 31, CR_ZR = 51, CR_Z = 71 };


// per-cell constants: active-face flags, g = d(grad p)/dp_c, P = I - g g^T/|g|^2
template <class S>
struct CellG {
  S act[4], g[4], gh[4], ig2;
  __device__ void init(const Geom& geo, int i, int j) {
    act[0] = S(i > 0);
    act[1] = S(i < geo.nx - 1);
    act[2] = S(j > 0);
    act[3] = S(j < geo.ny - 1);
    g[0] = act[0] * S(geo.ih);
    g[1] = -act[1] * S(geo.ih);
    g[2] = act[2] * S(geo.ih);
    g[3] = -act[3] * S(geo.ih);
    S g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + g[3] * g[3];
    ig2 = S(1) / g2;
#pragma unroll
    for (int a = 0; a < 4; ++a) gh[a] = g[a] * ig2;
  }
  // P w on the active faces (zero on inactive ones)
  __device__ __forceinline__ void proj(const S w[4], S out[4]) const {
    S d = g[0] * w[0] + g[1] * w[1] + g[2] * w[2] + g[3] * w[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) out[a] = act[a] * w[a] - gh[a] * d;
  }
};

template <class S>
__device__ __forceinline__ void load_sym(const S* v, S A[4][4]) {
  int e = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      A[a][b] = v[e];
      A[b][a] = v[e];
      ++e;
    }
}

template <class S>
__device__ __forceinline__ void store_sym(S* v, const S A[4][4]) {
  int e = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      v[e] = S(0.5) * (A[a][b] + A[b][a]);
      ++e;
    }
}

// shift A by gamma g g^T (gamma from the trace) and symmetrise; returns gamma
template <class S>
__device__ __forceinline__ S shift_sym(S A[4][4], const CellG<S>& cg) {
  S tr = A[0][0] + A[1][1] + A[2][2] + A[3][3];
  const S gam = S(0.25) * tr * cg.ig2;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      const S m = S(0.5) * (A[a][b] + A[b][a]) + gam * cg.g[a] * cg.g[b];
      A[a][b] = m;
      A[b][a] = m;
    }
  return gam;
}

// Shared-memory layout of the smoother: the U_t row of time t starts at t us,
// the b_u row at t bs (the entries of a row cpb apart, cells fastest), cell c's
// block records at c cs, block k of a cell at k STRIDE (+ k / 32 with shift).
// The warp kernel skews them so that a warp's lanes hit distinct banks: us and
// bs are = cpb (mod 32), so the lanes of a (cell, time) sweep read consecutive
// banks; cs is searched on the host; the one-word shift per 32 blocks parts the
// blocks 32 apart that lanes m and m + 16 of the reduction touch.
struct ScgsLay {
  int us, bs, cs, shift;
};

__host__ __device__ inline int blk_off(const ScgsLay& L, int k, int stride) {
  return k * stride + (L.shift ? k >> 5 : 0);
}

// Phases A and A2 of one colour's SCGS for the cells q0 .. q0 + cpb - 1 (see
// above): U_t, y_t and the v-block records (STRIDE values per block) in
// shared memory; ends with a CTA barrier.
template <class T, class S, int STRIDE>
__device__ __forceinline__ void scgs_assemble(const Geom& g, const State<T>& x, const CState<T>& r, int colour,
                                              int ncx, int ncell, int cpb, int q0, S lm, S* Us, S* Bu, S* Vb,
                                              const ScgsLay& L) {
  const int N = g.N;
  const S idt = pick<S>(g.idt, g.idtf);
  // ---- phase A: couplings and right-hand sides ----------------------------
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const int i = 2 * (q % ncx) + (colour & 1);
    const int j = 2 * (q / ncx) + (colour >> 1);
    const int fidx[4] = {xf(g, j, i), xf(g, j, i + 1), yf(g, j, i), yf(g, j + 1, i)};
    const T act[4] = {T(i > 0), T(i < g.nx - 1), T(j > 0), T(j < g.ny - 1)};
    const int cc = cidx(g, j, i);
    S Jl[4][4];   // in the solve type: the blocks are stored as S
    local_adv_jac<T, S>(g, x.v + (size_t)(t + 1) * g.F, j, i, Jl);
    S* U = Us + (size_t)t * L.us + c;
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2)
        U[(a2 * 4 + b2) * cpb] =
            ((a2 == b2 ? pick<S>(g.idt, g.idtf) : S(0)) + S(g.self_adv) * Jl[a2][b2]) * S(act[a2] * act[b2]);
    S* Ru = Bu + (size_t)t * L.bs + c;
    S* Rv = Vb + (size_t)c * L.cs + blk_off(L, t, STRIDE) + CR_R;
    const T* ru = r.u + (size_t)t * g.F;
    const T* rv = r.v + (size_t)(t + 1) * g.F;
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      Ru[a2 * cpb] = S(-ld(ru + fidx[a2]) * act[a2]);
      Rv[a2] = S(-ld(rv + fidx[a2]) * act[a2]);
    }
    Ru[4 * cpb] = S(-ld(r.p + (size_t)t * g.C + cc));
    Rv[4] = S(-ld(r.pbar + (size_t)(t + 1) * g.C + cc));
  }
  __syncthreads();

  // ---- phase A2: eliminate the u blocks ------------------------------------
  // (a) y_t = D_u^{-1} b_u(t) in place
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    CellG<S> cg_;
    cg_.init(g, 2 * (q % ncx) + (colour & 1), 2 * (q / ncx) + (colour >> 1));
    S* Ru = Bu + (size_t)t * L.bs + c;
    S bf[4], pb[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) bf[a2] = Ru[a2 * cpb];
    const S bp = Ru[4 * cpb];
    cg_.proj(bf, pb);
    S gb = S(0);
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) gb += cg_.gh[a2] * bf[a2];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) Ru[a2 * cpb] = -pb[a2] + cg_.gh[a2] * bp;
    Ru[4 * cpb] = gb + bp * cg_.ig2;
  }
  __syncthreads();
  // (b) v block j = t (v_{t+1}): S, R, and its upper coupling O_{t+1} = -P U_{t+1} / dt
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    CellG<S> cg_;
    cg_.init(g, 2 * (q % ncx) + (colour & 1), 2 * (q / ncx) + (colour >> 1));
    const int tv = t + 1;
    S* V = Vb + (size_t)c * L.cs + blk_off(L, t, STRIDE);
    const S* U = Us + (size_t)t * L.us + c;     // U_{tv-1}
    S Um[4][4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) Um[a2][b2] = U[(a2 * 4 + b2) * cpb];
    S PU[4][4];
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) {
      S w[4], pw[4];
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2) w[a2] = Um[a2][b2];
      cg_.proj(w, pw);
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2) PU[a2][b2] = pw[a2];
    }
    const S diag = (tv < N ? pick<S>(g.a, g.af) : S(0)) + lm;
    int e = 0;
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = a2; b2 < 4; ++b2) {
        S v = S(0);
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) v += Um[c2][a2] * PU[c2][b2];
        if (tv < N) v += ((a2 == b2 ? cg_.act[a2] : S(0)) - cg_.gh[a2] * cg_.g[b2]) * idt * idt;
        if (a2 == b2) v += cg_.act[a2] > S(0) ? diag : S(1);
        V[CR_A + e] = v;
        ++e;
      }
    // R = b_v + [tv<N] y_tv / dt - U_{tv-1}^T y_{tv-1}
    const S* y0 = Bu + (size_t)t * L.bs + c;
    S yv[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) yv[a2] = y0[a2 * cpb];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      S v = V[CR_R + a2];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) v -= Um[c2][a2] * yv[c2];
      if (tv < N) v += idt * cg_.act[a2] * Bu[(size_t)tv * L.bs + a2 * cpb + c];
      V[CR_R + a2] = v;
    }
    // coupling to v_{tv+1}: O_tv = -P U_tv / dt
    if (tv < N) {
      const S* U1 = Us + (size_t)tv * L.us + c;
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) {
        S w[4], pw[4];
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) w[a2] = U1[(a2 * 4 + b2) * cpb];
        cg_.proj(w, pw);
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) V[CR_C + a2 * 4 + b2] = -idt * pw[a2];
      }
    } else {
#pragma unroll
      for (int e2 = 0; e2 < 16; ++e2) V[CR_C + e2] = S(0);
    }
  }
  __syncthreads();

}

// Phase C: the u blocks from the solved v blocks, x += omega delta.
template <class T, class S, int STRIDE>
__device__ __forceinline__ void scgs_update(const Geom& g, const State<T>& x, int colour, int ncx, int ncell,
                                            int cpb, int q0, const S* Us, const S* Bu, const S* Vb,
                                            const ScgsLay& L) {
  const int N = g.N;
  const S idt = pick<S>(g.idt, g.idtf);
  // ---- phase C: u blocks from the v solution, x += omega * delta -----------
  // The old values of the 10 unknowns are all loaded before any store: the
  // state arrays may alias as far as the compiler knows, so interleaved
  // read-modify-writes would serialise ten global-memory latencies.
  const T om = pick<T>(g.omega, g.omegaf);
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const int i = 2 * (q % ncx) + (colour & 1);
    const int j = 2 * (q / ncx) + (colour >> 1);
    const int fidx[4] = {xf(g, j, i), xf(g, j, i + 1), yf(g, j, i), yf(g, j + 1, i)};
    const bool actb[4] = {i > 0, i < g.nx - 1, j > 0, j < g.ny - 1};
    const int cc = cidx(g, j, i);
    T* fu = x.u + (size_t)t * g.F;
    T* fv = x.v + (size_t)(t + 1) * g.F;
    T* fp = x.p + (size_t)t * g.C + cc;
    T* fpb = x.pbar + (size_t)(t + 1) * g.C + cc;
    T old_u[4], old_v[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      old_u[a2] = actb[a2] ? fu[fidx[a2]] : T(0);
      old_v[a2] = actb[a2] ? fv[fidx[a2]] : T(0);
    }
    const T old_p = *fp, old_pb = *fpb;
    CellG<S> cg_;
    cg_.init(g, i, j);
    // w = [t>=1] x_v(t)/dt - U_t x_v(t+1);  x_u = y_t + [-P w; gh^T w]
    const S* U = Us + (size_t)t * L.us + c;
    const S* xv1 = Vb + (size_t)c * L.cs + blk_off(L, t, STRIDE) + CR_Z;          // v_{t+1}
    const S* xv0 = Vb + (size_t)c * L.cs + blk_off(L, t > 0 ? t - 1 : 0, STRIDE) + CR_Z;   // v_t
    S w[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      S v = S(0);
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) v -= U[(a2 * 4 + b2) * cpb] * xv1[b2];
      if (t >= 1) v += idt * cg_.act[a2] * xv0[a2];
      w[a2] = v;
    }
    S pw[4];
    cg_.proj(w, pw);
    S gw = S(0);
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) gw += cg_.gh[a2] * w[a2];
    const S* y = Bu + (size_t)t * L.bs + c;
    S du[5];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) du[a2] = y[a2 * cpb] - pw[a2];
    du[4] = y[4 * cpb] + gw;
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
      if (actb[a2]) {
        fu[fidx[a2]] = old_u[a2] + om * T(du[a2]);
        fv[fidx[a2]] = old_v[a2] + om * T(xv1[a2]);
      }
    *fp = old_p + om * T(du[4]);
    *fpb = old_pb + om * T(xv1[4]);
  }
}

template <class T, class S>
__global__ void __launch_bounds__(256)
scgs_colour_kernel(Geom g, State<T> x, CState<T> r, int colour, int ncx, int ncy, int cpb,
                   const double* __restrict__ lm_dev, ScgsLay L) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.N;
  // Levenberg-Marquardt shift of the v blocks: a device scalar when the solve
  // adapts it between V-cycles (the captured graph stays valid), else g.lm
  const S lm = S(lm_dev ? *lm_dev : g.lm);
  const int ncell = ncx * ncy;
  const int q0 = blockIdx.x * cpb;
  S* Us = reinterpret_cast<S*>(smem_raw);            // U_t        [N][16][cpb], rows L.us apart
  S* Bu = Us + (size_t)N * L.us;                      // b_u -> y_t [N][5][cpb], rows L.bs apart
  S* Vb = Bu + (size_t)N * L.bs;                      // v blocks   [cpb][N][kCrStride], cells L.cs apart

  scgs_assemble<T, S, kCrStride>(g, x, r, colour, ncx, ncell, cpb, q0, lm, Us, Bu, Vb, L);

  // ---- phase B: cyclic reduction over the v blocks, one warp per cell -------
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = q0 + warp;
    if (warp < cpb && q < ncell) {
      CellG<S> cg_;
      cg_.init(g, 2 * (q % ncx) + (colour & 1), 2 * (q / ncx) + (colour >> 1));
      S* V = Vb + (size_t)warp * L.cs;
      int top = 0;
      for (int s2 = 1; s2 < N; s2 <<= 1) {
        top = s2;
        // eliminate the odd blocks o = s2 (2m + 1)
        for (int m = lane;; m += 32) {
          const int o = s2 * (2 * m + 1);
          if (o >= N) break;
          const bool hasb = o + s2 < N;
          S* Vo = V + blk_off(L, o, kCrStride);
          const S* Va = V + blk_off(L, o - s2, kCrStride);
          S A[4][4];
          load_sym(Vo + CR_A, A);
          S B[4][9];
          S qv[9];
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) {
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) {
              B[r2][c2] = Va[CR_C + c2 * 4 + r2];                  // (coupling a -> o)^T
              B[r2][4 + c2] = hasb ? Vo[CR_C + r2 * 4 + c2] : S(0);  // coupling o -> b
            }
            B[r2][8] = Vo[CR_R + r2];
          }
#pragma unroll
          for (int c2 = 0; c2 < 8; ++c2) qv[c2] = S(0);
          qv[8] = Vo[CR_R + 4];
          const S gam = shift_sym(A, cg_);
          S Y[9];
          saddle_solve<S, 9>(A, cg_.g, B, qv, Y);
          Y[8] += gam * qv[8];
#pragma unroll
          for (int c2 = 0; c2 < 4; ++c2) {
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2) {
              Vo[CR_ZL + r2 * 4 + c2] = B[r2][c2];
              Vo[CR_ZR + r2 * 4 + c2] = B[r2][4 + c2];
            }
            Vo[CR_ZL + 16 + c2] = Y[c2];
            Vo[CR_ZR + 16 + c2] = Y[4 + c2];
          }
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) Vo[CR_Z + r2] = B[r2][8];
          Vo[CR_Z + 4] = Y[8];
        }
        __syncwarp();
        // update the even blocks e = 2 s2 m from both eliminated neighbours
        for (int m = lane;; m += 32) {
          const int e = 2 * s2 * m;
          if (e >= N) break;
          S* Ve = V + blk_off(L, e, kCrStride);
          S A[4][4];
          load_sym(Ve + CR_A, A);
          S rf[4], Ce[4][4], Cn[4][4];
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) {
            rf[r2] = Ve[CR_R + r2];
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) {
              Ce[r2][c2] = Ve[CR_C + r2 * 4 + c2];
              Cn[r2][c2] = S(0);
            }
          }
          const int o2 = e + s2;
          if (o2 < N) {
            const S* V2 = V + blk_off(L, o2, kCrStride);
            const bool hasb2 = o2 + s2 < N;
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2) {
#pragma unroll
              for (int c2 = 0; c2 < 4; ++c2) {
                S aL = S(0), aR = S(0);
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) {
                  aL += Ce[r2][k2] * V2[CR_ZL + k2 * 4 + c2];
                  aR += Ce[r2][k2] * V2[CR_ZR + k2 * 4 + c2];
                }
                A[r2][c2] -= aL;
                Cn[r2][c2] = hasb2 ? -aR : S(0);
              }
              S az = S(0);
#pragma unroll
              for (int k2 = 0; k2 < 4; ++k2) az += Ce[r2][k2] * V2[CR_Z + k2];
              rf[r2] -= az;
            }
          }
          const int o1 = e - s2;
          if (o1 >= 0) {
            const S* V1 = V + blk_off(L, o1, kCrStride);
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2) {
#pragma unroll
              for (int c2 = 0; c2 < 4; ++c2) {
                S aR = S(0);
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) aR += V1[CR_C + k2 * 4 + r2] * V1[CR_ZR + k2 * 4 + c2];
                A[r2][c2] -= aR;
              }
              S az = S(0);
#pragma unroll
              for (int k2 = 0; k2 < 4; ++k2) az += V1[CR_C + k2 * 4 + r2] * V1[CR_Z + k2];
              rf[r2] -= az;
            }
          }
          store_sym(Ve + CR_A, A);
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) {
            Ve[CR_R + r2] = rf[r2];
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) Ve[CR_C + r2 * 4 + c2] = Cn[r2][c2];
          }
        }
        __syncwarp();
      }
      // the last remaining block
      if (lane == 0) {
        S A[4][4];
        load_sym(V + CR_A, A);
        S B[4][1];
        S qv[1] = {V[CR_R + 4]};
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) B[r2][0] = V[CR_R + r2];
        const S gam = shift_sym(A, cg_);
        S Y[1];
        saddle_solve<S, 1>(A, cg_.g, B, qv, Y);
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) V[CR_Z + r2] = B[r2][0];
        V[CR_Z + 4] = Y[0] + gam * qv[0];
      }
      __syncwarp();
      // unwind: x_o = z_o - ZL_o x_a - ZR_o x_b (faces of the neighbours)
      for (int s2 = top; s2 >= 1; s2 >>= 1) {
        for (int m = lane;; m += 32) {
          const int o = s2 * (2 * m + 1);
          if (o >= N) break;
          S* Vo = V + blk_off(L, o, kCrStride);
          const S* Va = V + blk_off(L, o - s2, kCrStride);
          const bool hasb = o + s2 < N;
          S xa[4], xb[4];
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) {
            xa[k2] = Va[CR_Z + k2];
            xb[k2] = hasb ? V[blk_off(L, o + s2, kCrStride) + CR_Z + k2] : S(0);
          }
#pragma unroll
          for (int r2 = 0; r2 < 5; ++r2) {
            S v = Vo[CR_Z + r2];
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v -= Vo[CR_ZL + r2 * 4 + k2] * xa[k2] + Vo[CR_ZR + r2 * 4 + k2] * xb[k2];
            Vo[CR_Z + r2] = v;
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();

  scgs_update<T, S, kCrStride>(g, x, colour, ncx, ncell, cpb, q0, Us, Bu, Vb, L);
}

// The same colour step with one CTA per cell, for colours of few cells (the
// coarse levels), where the warp-per-cell reduction leaves the GPU idle and
// its time is the length of one cell's dependency chain.  Every block step of
// the cyclic reduction is split over the CTA's threads: an odd block's
// elimination by right-hand-side column (each thread a saddle solve with one
// column: the same factorisation and the same arithmetic per column as the
// nine-column solve), an even block's update by output entry (the 10 entries
// of the symmetric face block, 4 of the right-hand side, 16 of the new
// coupling), the unwinding by unknown.  The couplings are double-buffered
// (CR_C at even levels, CR_C2 at odd ones) because an even block's update
// reads its old coupling while writing the new one.
constexpr int kCrStride2 = 93;
enum : int { CR_C2 = 77 };
// threads of the CTA-per-cell kernel: 256 on colours of at most 256 cells
// (shorter rounds of the split block steps), 128 on larger ones (occupancy)
constexpr int kCellCtaThreadsSmall = 256, kCellCtaThreadsLarge = 128, kCellCtaSmallCells = 256;

// (U rows 17 apart: odd, so the time-indexed lanes of a one-cell CTA hit distinct banks)
__host__ __device__ inline size_t scgs_cell_floats2(int N) { return (size_t)(17 + 5 + kCrStride2) * N; }

template <bool WARP>
__device__ __forceinline__ void group_sync() {
  if (WARP) __syncwarp();
  else __syncthreads();
}

// The split cyclic reduction of one cell's v blocks V (records of kCrStride2)
// by a group of nl threads (rank lane): a warp (WARP) or the whole CTA.  (A
// warp per cell with this split measured slower than the nine-column solve
// per lane at every level: the split repeats the factorisation per column and
// its task kinds diverge within the warp; only a CTA per cell gains.)
template <class S, bool WARP>
__device__ __forceinline__ void cr_split(S* V, int N, const CellG<S>& cg_, int lane, int nl) {
  int top = 0, lev = 0;
  for (int s2 = 1; s2 < N; s2 <<= 1, ++lev) {
    top = s2;
    const int cur = (lev & 1) ? CR_C2 : CR_C, nxt = (lev & 1) ? CR_C : CR_C2;
    const int nk = (N + s2 - 1) / s2;      // blocks k s2 < N; odd k are eliminated
    const int nodd = nk / 2, neven = (nk + 1) / 2;
    // eliminate the odd blocks o = s2 (2m + 1), one right-hand-side column per thread
    for (int task = lane; task < nodd * 9; task += nl) {
      const int m = task / 9, col = task - 9 * m;
      const int o = s2 * (2 * m + 1);
      const bool hasb = o + s2 < N;
      S* Vo = V + (size_t)o * kCrStride2;
      const S* Va = V + (size_t)(o - s2) * kCrStride2;
      S A[4][4];
      load_sym(Vo + CR_A, A);
      S B[4][1];
#pragma unroll
      for (int r2 = 0; r2 < 4; ++r2)
        B[r2][0] = col < 4 ? Va[cur + col * 4 + r2]                                  // (coupling a -> o)^T
                 : col < 8 ? (hasb ? Vo[cur + r2 * 4 + (col - 4)] : S(0))           // coupling o -> b
                           : Vo[CR_R + r2];
      S qv[1] = {col == 8 ? Vo[CR_R + 4] : S(0)};
      const S gam = shift_sym(A, cg_);
      S Y[1];
      saddle_solve<S, 1>(A, cg_.g, B, qv, Y);
      if (col < 8) {
        S* Z = Vo + (col < 4 ? CR_ZL : CR_ZR);
        const int c2 = col & 3;
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) Z[r2 * 4 + c2] = B[r2][0];
        Z[16 + c2] = Y[0];
      } else {
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) Vo[CR_Z + r2] = B[r2][0];
        Vo[CR_Z + 4] = Y[0] + gam * qv[0];
      }
    }
    group_sync<WARP>();
    // update the even blocks e = 2 s2 m from both eliminated neighbours, one entry per thread
    for (int task = lane; task < neven * 30; task += nl) {
      const int m = task / 30, k = task - 30 * m;
      const int e = 2 * s2 * m;
      S* Ve = V + (size_t)e * kCrStride2;
      const int o2 = e + s2, o1 = e - s2;
      const S* V2 = o2 < N ? V + (size_t)o2 * kCrStride2 : nullptr;
      const S* V1 = o1 >= 0 ? V + (size_t)o1 * kCrStride2 : nullptr;
      if (k < 10) {
        // A[a][b] and A[b][a] as the warp kernel forms them, then symmetrised
        // row a, column b of the k-th stored entry (rows of the upper triangle)
        const int a = k < 4 ? 0 : k < 7 ? 1 : k < 9 ? 2 : 3;
        const int b = k < 4 ? k : k < 7 ? k - 3 : k < 9 ? k - 5 : 3;
        S ab = Ve[CR_A + k], ba = ab;
        if (V2) {
          S aL = S(0), bL = S(0);
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) {
            aL += Ve[cur + a * 4 + k2] * V2[CR_ZL + k2 * 4 + b];
            bL += Ve[cur + b * 4 + k2] * V2[CR_ZL + k2 * 4 + a];
          }
          ab -= aL;
          ba -= bL;
        }
        if (V1) {
          S aR = S(0), bR = S(0);
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) {
            aR += V1[cur + k2 * 4 + a] * V1[CR_ZR + k2 * 4 + b];
            bR += V1[cur + k2 * 4 + b] * V1[CR_ZR + k2 * 4 + a];
          }
          ab -= aR;
          ba -= bR;
        }
        Ve[CR_A + k] = S(0.5) * (ab + ba);
      } else if (k < 14) {
        const int r2 = k - 10;
        S rf = Ve[CR_R + r2];
        if (V2) {
          S az = S(0);
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) az += Ve[cur + r2 * 4 + k2] * V2[CR_Z + k2];
          rf -= az;
        }
        if (V1) {
          S az = S(0);
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) az += V1[cur + k2 * 4 + r2] * V1[CR_Z + k2];
          rf -= az;
        }
        Ve[CR_R + r2] = rf;
      } else {
        const int r2 = (k - 14) >> 2, c2 = (k - 14) & 3;
        S cn = S(0);
        if (V2 && o2 + s2 < N) {
          S aR = S(0);
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) aR += Ve[cur + r2 * 4 + k2] * V2[CR_ZR + k2 * 4 + c2];
          cn = -aR;
        }
        Ve[nxt + r2 * 4 + c2] = cn;
      }
    }
    group_sync<WARP>();
  }
  // the last remaining block
  if (lane == 0) {
    S A[4][4];
    load_sym(V + CR_A, A);
    S B[4][1];
    S qv[1] = {V[CR_R + 4]};
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) B[r2][0] = V[CR_R + r2];
    const S gam = shift_sym(A, cg_);
    S Y[1];
    saddle_solve<S, 1>(A, cg_.g, B, qv, Y);
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) V[CR_Z + r2] = B[r2][0];
    V[CR_Z + 4] = Y[0] + gam * qv[0];
  }
  group_sync<WARP>();
  // unwind: x_o = z_o - ZL_o x_a - ZR_o x_b, one unknown per thread
  for (int s2 = top; s2 >= 1; s2 >>= 1) {
    const int nodd = ((N + s2 - 1) / s2) / 2;
    for (int task = lane; task < nodd * 5; task += nl) {
      const int m = task / 5, r2 = task - 5 * m;
      const int o = s2 * (2 * m + 1);
      S* Vo = V + (size_t)o * kCrStride2;
      const S* Va = V + (size_t)(o - s2) * kCrStride2;
      const bool hasb = o + s2 < N;
      S v = Vo[CR_Z + r2];
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) {
        const S xb = hasb ? V[(size_t)(o + s2) * kCrStride2 + CR_Z + k2] : S(0);
        v -= Vo[CR_ZL + r2 * 4 + k2] * Va[CR_Z + k2] + Vo[CR_ZR + r2 * 4 + k2] * xb;
      }
      Vo[CR_Z + r2] = v;
    }
    group_sync<WARP>();
  }
}

template <class T, class S, int THREADS>
__global__ void __launch_bounds__(THREADS)
scgs_colour_cell_kernel(Geom g, State<T> x, CState<T> r, int colour, int ncx, int ncy,
                        const double* __restrict__ lm_dev) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.N;
  const S lm = S(lm_dev ? *lm_dev : g.lm);
  const int ncell = ncx * ncy;
  const int q = blockIdx.x;
  S* Us = reinterpret_cast<S*>(smem_raw);            // U_t        [N][17] (16 used)
  S* Bu = Us + (size_t)N * 17;                        // b_u -> y_t [N][5]
  S* V = Bu + (size_t)N * 5;                          // v blocks   [N][kCrStride2]
  const ScgsLay L{17, 5, N * kCrStride2, 0};
  scgs_assemble<T, S, kCrStride2>(g, x, r, colour, ncx, ncell, 1, q, lm, Us, Bu, V, L);

  CellG<S> cg_;
  cg_.init(g, 2 * (q % ncx) + (colour & 1), 2 * (q / ncx) + (colour >> 1));
  cr_split<S, false>(V, N, cg_, threadIdx.x, blockDim.x);
  scgs_update<T, S, kCrStride2>(g, x, colour, ncx, ncell, 1, q, Us, Bu, V, L);
}

// ---------------------------------------------------------------------------
// transfers (Sec. 4.3): R = mean of the 4 children (cells) / the 2 coincident
// fine faces (faces); P = bilinear interpolation, faces linear along the
// normal and (3/4, 1/4) across, clamped at walls.
// ---------------------------------------------------------------------------
// Time modes of the transfers (levels that also halve N, an opt-in):
//   0  slab t <-> slab t (space-only hierarchy)
//   1  point fields (v, pbar, their rows): injection at the first and last
//      point, full weighting (1/4, 1/2, 1/4) inside; prolongation linear
//   2  interval fields (u, p, their rows): mean of the two sub-intervals;
//      prolongation piecewise constant
//   3  the targets z_0..z_{N-1}: injection at 0, full weighting after
// The spatial transfer is applied per slab, then the time weights.
template <class Tf, class Tc>
__global__ void restrict_kernel(Geom gf, Geom gc, int nt_face, int nt_cell, const Tf* __restrict__ sf,
                                const Tf* __restrict__ sc_cells, Tc* df, Tc* dc_cells, Tc* df2,
                                Tc* dc2, int tmode) {
  pdl_wait();
  // faces: nt_face coarse slabs of gc.F entries; cells: nt_cell coarse slabs of gc.C
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nfaces = (size_t)nt_face * gc.F;
  const size_t ncells = (size_t)nt_cell * gc.C;
  auto in_time = [&](auto rs, int t, int nt) -> Tc {
    switch (tmode) {
      case 0: return rs(t);
      case 1:
        if (t == 0 || t == nt - 1) return rs(2 * t);
        return Tc(0.25) * rs(2 * t - 1) + Tc(0.5) * rs(2 * t) + Tc(0.25) * rs(2 * t + 1);
      case 2: return Tc(0.5) * (rs(2 * t) + rs(2 * t + 1));
      default:
        if (t == 0) return rs(0);
        return Tc(0.25) * rs(2 * t - 1) + Tc(0.5) * rs(2 * t) + Tc(0.25) * rs(2 * t + 1);
    }
  };
  if (e < nfaces) {
    const int t = (int)(e / gc.F);
    const int f = (int)(e - (size_t)t * gc.F);
    auto rs = [&](int tf) -> Tc {
      const Tf* s = sf + (size_t)tf * gf.F;
      if (f < gc.Fx) {
        int J = f / (gc.nx + 1), I = f - J * (gc.nx + 1);
        return Tc(0.5) * (Tc(s[xf(gf, 2 * J, 2 * I)]) + Tc(s[xf(gf, 2 * J + 1, 2 * I)]));
      }
      int q = f - gc.Fx;
      int J = q / gc.nx, I = q - J * gc.nx;
      return Tc(0.5) * (Tc(s[yf(gf, 2 * J, 2 * I)]) + Tc(s[yf(gf, 2 * J, 2 * I + 1)]));
    };
    const Tc val = in_time(rs, t, nt_face);
    df[e] = val;
    if (df2) df2[e] = val;
  } else if (e < nfaces + ncells) {
    const size_t ec = e - nfaces;
    const int t = (int)(ec / gc.C);
    const int c = (int)(ec - (size_t)t * gc.C);
    const int J = c / gc.nx, I = c - J * gc.nx;
    auto rs = [&](int tf) -> Tc {
      const Tf* s = sc_cells + (size_t)tf * gf.C;
      return Tc(0.25) * (Tc(s[cidx(gf, 2 * J, 2 * I)]) + Tc(s[cidx(gf, 2 * J, 2 * I + 1)]) +
                         Tc(s[cidx(gf, 2 * J + 1, 2 * I)]) + Tc(s[cidx(gf, 2 * J + 1, 2 * I + 1)]));
    };
    const Tc val = in_time(rs, t, nt_cell);
    dc_cells[ec] = val;
    if (dc2) dc2[ec] = val;
  }
}

__device__ __forceinline__ void cell_interp(int k, int nc, int& a, int& b) {
  a = k >> 1;
  b = (k & 1) ? a + 1 : a - 1;
  b = b < 0 ? 0 : (b > nc - 1 ? nc - 1 : b);
}

// fine += P(coarse_new - coarse_old) for faces (t in [t0, t0+nt)) and cells
template <class Tf, class Tc>
__global__ void prolong_correct_kernel(Geom gf, Geom gc, int nt_face, int nt_cell, int t0_face,
                                       int t0_cell, Tf* ff, Tf* fc, const Tc* __restrict__ cnf,
                                       const Tc* __restrict__ cof, const Tc* __restrict__ cnc,
                                       const Tc* __restrict__ coc, const double* undo_if_rose, int tmode) {
  pdl_wait();
  // undo form: subtract the same correction again when the guarded level's
  // residual norm rose (norms[1] after vs norms[0] before; NaN counts as rose)
  // interpolation arithmetic: fp64 when either level is fp64, else fp32
  using W = typename std::conditional<(sizeof(Tf) == 8 || sizeof(Tc) == 8), double, float>::type;
  W sgn = W(1);
  if (undo_if_rose) {
    if (undo_if_rose[1] <= undo_if_rose[0]) return;
    sgn = W(-1);
  }
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nfaces = (size_t)nt_face * gf.F;
  const size_t ncells = (size_t)nt_cell * gf.C;
  // fine slab t of the correction from the coarse slab(s) it sits on (time modes
  // as in restrict_kernel: 1 linear between points, 2 piecewise constant)
  auto in_time = [&](auto ps, int t) -> W {
    if (tmode == 0) return ps(t);
    if (tmode == 2) return ps(t >> 1);
    if ((t & 1) == 0) return ps(t >> 1);
    return W(0.5) * (ps(t >> 1) + ps((t >> 1) + 1));
  };
  if (e < nfaces) {
    const int t = (int)(e / gf.F) + t0_face;
    const int f = (int)(e - (size_t)(t - t0_face) * gf.F);
    auto ps = [&](int tc) -> W {
    const Tc* n = cnf + (size_t)tc * gc.F;
    const Tc* o = cof + (size_t)tc * gc.F;
    W val;
    if (f < gf.Fx) {
      int j = f / (gf.nx + 1), i = f - j * (gf.nx + 1);
      int ja, jb;
      cell_interp(j, gc.ny, ja, jb);
      int ia = i >> 1, ib = (i & 1) ? ia + 1 : ia;
      W wb = (i & 1) ? W(0.5) : W(0), wa = W(1) - wb;
      auto d = [&](int J, int I) { return W(n[xf(gc, J, I)]) - W(o[xf(gc, J, I)]); };
      W ta = W(0.75) * d(ja, ia) + W(0.25) * d(jb, ia);
      W tb = W(0.75) * d(ja, ib) + W(0.25) * d(jb, ib);
      val = wa * ta + wb * tb;
    } else {
      int qq = f - gf.Fx;
      int j = qq / gf.nx, i = qq - j * gf.nx;
      int ia, ib;
      cell_interp(i, gc.nx, ia, ib);
      int ja = j >> 1, jb = (j & 1) ? ja + 1 : ja;
      W wb = (j & 1) ? W(0.5) : W(0), wa = W(1) - wb;
      auto d = [&](int J, int I) { return W(n[yf(gc, J, I)]) - W(o[yf(gc, J, I)]); };
      W ta = W(0.75) * d(ja, ia) + W(0.25) * d(ja, ib);
      W tb = W(0.75) * d(jb, ia) + W(0.25) * d(jb, ib);
      val = wa * ta + wb * tb;
    }
    return val;
    };
    ff[(size_t)t * gf.F + f] += Tf(sgn * in_time(ps, t));
  } else if (e < nfaces + ncells) {
    const size_t ec = e - nfaces;
    const int t = (int)(ec / gf.C) + t0_cell;
    const int c = (int)(ec - (size_t)(t - t0_cell) * gf.C);
    int j = c / gf.nx, i = c - j * gf.nx;
    int ja, jb, ia, ib;
    cell_interp(j, gc.ny, ja, jb);
    cell_interp(i, gc.nx, ia, ib);
    auto ps = [&](int tc) -> W {
      const Tc* n = cnc + (size_t)tc * gc.C;
      const Tc* o = coc + (size_t)tc * gc.C;
      auto d = [&](int J, int I) { return W(n[cidx(gc, J, I)]) - W(o[cidx(gc, J, I)]); };
      return W(0.5625) * d(ja, ia) + W(0.1875) * d(ja, ib) + W(0.1875) * d(jb, ia) + W(0.0625) * d(jb, ib);
    };
    fc[(size_t)t * gf.C + c] += Tf(sgn * in_time(ps, t));
  }
}

// ---------------------------------------------------------------------------
// reductions (fp64) and small elementwise kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// max |a| into *out (fp64) and a flag for non-finite entries.  A max is exact
// in the element type: the reduction runs in T and converts once per block.
template <class T>
__global__ void absmax_kernel(const T* __restrict__ a, size_t n, double* out, int* err) {
  pdl_wait();
  T m = T(0);
  bool bad = false;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const T v = fabs(a[e]);
    if (!isfinite(v)) bad = true;
    else m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ T sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x + 31) / 32) ? sm[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomic_max_nonneg(out, (double)m);
  }
  if (bad && err) atomicOr(err, DEV_NONFINITE);
}

template <class T>
__global__ void sumsq_kernel(const T* __restrict__ a, size_t n, double* out, RedScratch rs) {
  pdl_wait();
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = (double)a[e];
    s += v * v;
  }
  block_sum_ordered(s, out, rs);
}

// subtract the mean of each of `count` slabs of length C (one block per slab)
template <class T>
__global__ void remove_mean_kernel(T* a, int C) {
  pdl_wait();
  T* s = a + (size_t)blockIdx.x * C;
  double acc = 0.0;
  for (int e = threadIdx.x; e < C; e += blockDim.x) acc += (double)s[e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double sm[32];
  __shared__ double mean;
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) tot += sm[w];
    mean = tot / C;
  }
  __syncthreads();
  const T m = T(mean);
  for (int e = threadIdx.x; e < C; e += blockDim.x) s[e] -= m;
}

template <class Ts, class Td>
__global__ void convert_kernel(const Ts* __restrict__ s, Td* d, size_t n) {
  pdl_wait();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    d[e] = Td(s[e]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// Launch with the programmatic-stream-serialization attribute (see pdl_wait):
// inside the captured V-cycle graph consecutive kernels get programmatic
// edges, so a kernel's launch overlaps the end of its predecessor.
template <class... KArgs, class... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <class T>
int launch_nso_residual(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, T sf, T sr,
                        cudaStream_t st, double* sq, const double* only_if_undone, RedScratch rs, void* lamb,
                        size_t lamb_bytes) {
  if (g.dim == 3)
    return launch_nso_residual3<T>(g, x, z, res, out, sf, sr, st, sq, only_if_undone, rs, lamb, lamb_bytes);
  const int tpb = 128;
  const int n = g.F > g.C ? g.F : g.C;
  dim3 grid(blocks_for(n, tpb), g.N + 1);
  launch_pdl(nso_residual_kernel<T>, grid, dim3(tpb), 0, st, g, x, z, res, out, sf, sr, sq, rs, only_if_undone);
  return 1;
}

size_t nso_residual_blocks(const Geom& g) {
  if (g.dim == 3) return nso_residual3_blocks(g);
  const int n = g.F > g.C ? g.F : g.C;
  return (size_t)blocks_for(n, 128) * (g.N + 1);
}

int colour_extent(int n, int parity) { return (n - parity + 1) / 2; }

template <class T>
int launch_nso_residual_colour(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, int colour,
                               cudaStream_t st, const double* only_if_undone, void* lamb, size_t lamb_bytes) {
  if (g.dim == 3) return launch_nso_residual3_colour<T>(g, x, z, res, out, colour, st, only_if_undone, lamb, lamb_bytes);
  const int px = colour & 1, py = colour >> 1;
  const int nrx = colour_extent(g.ny, py), ncy = colour_extent(g.nx, px);
  const int n = nrx * (g.nx + 1) + (g.ny + 1) * ncy + colour_extent(g.nx, px) * nrx;
  const int tpb = 128;
  dim3 grid(blocks_for(n, tpb), g.N + 1);
  launch_pdl(nso_residual_colour_kernel<T>, grid, dim3(tpb), 0, st, g, x, z, res, out, px, py, only_if_undone);
  return 1;
}

// the warp kernel's skewed layout for N blocks and cpb cells per CTA; cs is the
// first stride from the dense size whose (cell, time) sweep has the fewest
// lanes per bank (a constant offset rotates the banks, so one offset suffices)
ScgsLay scgs_warp_layout(int N, int cpb) {
  auto skew = [](int x, int m) { return x + (((m - x) % 32) + 32) % 32; };
  ScgsLay L;
  L.us = skew(16 * cpb, cpb);
  L.bs = skew(5 * cpb, cpb);
  L.shift = 1;
  const int base = N * kCrStride + ((N - 1) >> 5) + 1;
  L.cs = base;
  int best = 1 << 30;
  for (int cs = base; cs < base + 32; ++cs) {
    int cnt[32] = {0}, worst = 0;
    for (int l = 0; l < 32 && l / cpb < N; ++l) {
      const int bank = (int)(((long long)(l % cpb) * cs + blk_off(L, l / cpb, kCrStride)) % 32);
      worst = std::max(worst, ++cnt[bank]);
    }
    if (worst < best) {
      best = worst;
      L.cs = cs;
    }
  }
  return L;
}

struct WarpPlan {
  int cpb;
  ScgsLay lay;
  size_t bytes;
};

static size_t scgs_warp_bytes(int N, int cpb, const ScgsLay& L, size_t tsize) {
  return ((size_t)N * (L.us + L.bs) + (size_t)cpb * L.cs) * tsize;
}

// one warp per cell, at most 8 per CTA, two CTAs per SM (228 KB of shared
// memory per SM, 1 KB of it reserved per CTA), in the skewed layout; when not
// even one cell fits that way (long horizons: the skew pads a one-cell row of
// b_u from 5 to 33 values), one cell per CTA in the dense layout (U rows 17
// apart, b_u rows 5: odd, so the time-indexed lanes still hit distinct banks)
template <class S>
WarpPlan scgs_warp_plan(int N) {
  for (int c = 8; c >= 1; --c) {
    const ScgsLay L = scgs_warp_layout(N, c);
    const size_t b = scgs_warp_bytes(N, c, L, sizeof(S));
    if (b <= 115712) return {c, L, b};
  }
  const ScgsLay L{17, 5, N * kCrStride + ((N - 1) >> 5) + 1, 1};
  return {1, L, scgs_warp_bytes(N, 1, L, sizeof(S))};
}

// the CTA-per-cell kernel with THREADS threads (false: the records do not fit)
template <class T, class S, int THREADS>
static bool launch_scgs_cell_tts(const Geom& g, State<T> x, CState<T> r, int colour, int ncx, int ncy,
                                 const double* lm_dev, cudaStream_t st) {
  static std::once_flag attr_once;
  static int max_smem = 0;
  std::call_once(attr_once, [] {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, (const void*)scgs_colour_cell_kernel<T, S, THREADS>);
    max_smem = 227 * 1024 - (int)fa.sharedSizeBytes;
    cudaFuncSetAttribute((const void*)scgs_colour_cell_kernel<T, S, THREADS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  });
  const size_t sm = scgs_cell_floats2(g.N) * sizeof(S);
  if (sm > (size_t)max_smem) return false;
  launch_pdl(scgs_colour_cell_kernel<T, S, THREADS>, dim3(ncx * ncy), dim3(THREADS), sm, st, g, x, r, colour, ncx,
             ncy, lm_dev);
  return true;
}

// the CTA-per-cell kernel; false (nothing launched) when one cell's records
// do not fit in shared memory
template <class T, class S>
static bool launch_scgs_cell_ts(const Geom& g, State<T> x, CState<T> r, int colour, int ncx, int ncy,
                                const double* lm_dev, cudaStream_t st) {
  if (ncx * ncy <= kCellCtaSmallCells)
    return launch_scgs_cell_tts<T, S, kCellCtaThreadsSmall>(g, x, r, colour, ncx, ncy, lm_dev, st);
  return launch_scgs_cell_tts<T, S, kCellCtaThreadsLarge>(g, x, r, colour, ncx, ncy, lm_dev, st);
}

template <class T, class S>
static void launch_scgs_ts(const Geom& g, State<T> x, CState<T> r, int colour, const double* lm_dev,
                           cudaStream_t st) {
  const int ncx = colour_extent(g.nx, colour & 1);
  const int ncy = colour_extent(g.ny, colour >> 1);
  const int ncell = ncx * ncy;
  if (ncell <= 0) return;
  // measured on the 128^2 x 40 hierarchy: fp32 solves are faster with a warp
  // per cell above ~256 cells per colour, fp64 solves with a CTA per cell at
  // every level
  const int cta_cells = g.cta_cells >= 0 ? g.cta_cells : (sizeof(S) == 4 ? 256 : 1 << 30);
  if (ncell <= cta_cells && launch_scgs_cell_ts<T, S>(g, x, r, colour, ncx, ncy, lm_dev, st)) return;
  const WarpPlan plan = scgs_warp_plan<S>(g.N);
  const int cpb = plan.cpb;
  const ScgsLay lay = plan.lay;
  const size_t sm = plan.bytes;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, (const void*)scgs_colour_kernel<T, S>);
    cudaFuncSetAttribute((const void*)scgs_colour_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024 - (int)fa.sharedSizeBytes);
  });
  launch_pdl(scgs_colour_kernel<T, S>, dim3(blocks_for(ncell, cpb)), dim3(32 * cpb), sm, st, g, x, r, colour, ncx, ncy,
             cpb, lm_dev, lay);
}

template <class T>
int launch_scgs_colour(const Geom& g, State<T> x, CState<T> r, int colour, bool solve_fp32, cudaStream_t st,
                       const double* lm_dev, void* scratch3) {
  if (g.dim == 3) return launch_scgs3_colour<T>(g, x, r, colour, solve_fp32, st, lm_dev, scratch3);
  if (solve_fp32) launch_scgs_ts<T, float>(g, x, r, colour, lm_dev, st);
  else launch_scgs_ts<T, T>(g, x, r, colour, lm_dev, st);
  return 1;
}

size_t scgs_smem_bytes(int N, size_t tsize) {
  return tsize == 4 ? scgs_warp_plan<float>(N).bytes : scgs_warp_plan<double>(N).bytes;
}

template <class Tf, class Tc>
void launch_restrict(const Geom& gf, const Geom& gc, CState<Tf> s, State<Tc> d, State<Tc> d2, cudaStream_t st) {
  if (gf.dim == 3) return launch_restrict3<Tf, Tc>(gf, gc, s, d, d2, st);
  const int tpb = 256;
  const int N = gc.N;                       // coarse slab counts
  const bool in_time = gc.N != gf.N;
  // v (N+1 slabs) with pbar (N+1), then u (N) with p (N)
  size_t n1 = (size_t)(N + 1) * gc.F + (size_t)(N + 1) * gc.C;
  launch_pdl(restrict_kernel<Tf, Tc>, dim3(blocks_for(n1, tpb)), dim3(tpb), 0, st, gf, gc, N + 1, N + 1, s.v, s.pbar,
             d.v, d.pbar, d2.v, d2.pbar, in_time ? 1 : 0);
  size_t n2 = (size_t)N * gc.F + (size_t)N * gc.C;
  launch_pdl(restrict_kernel<Tf, Tc>, dim3(blocks_for(n2, tpb)), dim3(tpb), 0, st, gf, gc, N, N, s.u, s.p, d.u, d.p,
             d2.u, d2.p, in_time ? 2 : 0);
}

template <class Tf, class Tc>
void launch_restrict_faces(const Geom& gf, const Geom& gc, int nt, const Tf* s, Tc* d, cudaStream_t st) {
  if (gf.dim == 3) return launch_restrict3_faces<Tf, Tc>(gf, gc, nt, s, d, st);
  const int tpb = 256;
  // nt fine target slabs; the coarse level holds nt / 2 of them when it halves N
  const bool in_time = gc.N != gf.N;
  const int ntc = in_time ? nt / 2 : nt;
  size_t n = (size_t)ntc * gc.F;
  launch_pdl(restrict_kernel<Tf, Tc>, dim3(blocks_for(n, tpb)), dim3(tpb), 0, st, gf, gc, ntc, 0, s,
             (const Tf*)nullptr, d, (Tc*)nullptr, (Tc*)nullptr, (Tc*)nullptr, in_time ? 3 : 0);
}

template <class Tf, class Tc>
void launch_prolong_correct(const Geom& gf, const Geom& gc, State<Tf> f, CState<Tc> cn, CState<Tc> co,
                            cudaStream_t st, const double* undo_if_rose) {
  if (gf.dim == 3) return launch_prolong3_correct<Tf, Tc>(gf, gc, f, cn, co, st, undo_if_rose);
  const int tpb = 256;
  const int N = gf.N;
  const bool in_time = gc.N != gf.N;
  // v and pbar for t = 1..N (v_0 is data), u and p for t = 0..N-1
  size_t n1 = (size_t)N * gf.F + (size_t)N * gf.C;
  launch_pdl(prolong_correct_kernel<Tf, Tc>, dim3(blocks_for(n1, tpb)), dim3(tpb), 0, st, gf, gc, N, N, 1, 1, f.v,
             f.pbar, cn.v, co.v, cn.pbar, co.pbar, undo_if_rose, in_time ? 1 : 0);
  size_t n2 = (size_t)N * gf.F + (size_t)N * gf.C;
  launch_pdl(prolong_correct_kernel<Tf, Tc>, dim3(blocks_for(n2, tpb)), dim3(tpb), 0, st, gf, gc, N, N, 0, 0, f.u,
             f.p, cn.u, co.u, cn.p, co.p, undo_if_rose, in_time ? 2 : 0);
}

template <class T>
void launch_absmax(const T* a, size_t n, double* out, int* err, cudaStream_t st) {
  const int tpb = 256;
  unsigned nb = blocks_for(n, tpb);
  if (nb > 1216) nb = 1216;
  if (nb == 0) nb = 1;
  launch_pdl(absmax_kernel<T>, dim3(nb), dim3(tpb), 0, st, a, n, out, err);
}

template <class T>
void launch_sumsq(const T* a, size_t n, double* out, cudaStream_t st, RedScratch rs) {
  const int tpb = 256;
  unsigned nb = blocks_for(n, tpb);
  if (nb > kReduceMaxBlocks) nb = kReduceMaxBlocks;
  if (nb == 0) nb = 1;
  launch_pdl(sumsq_kernel<T>, dim3(nb), dim3(tpb), 0, st, a, n, out, rs);
}

template <class T>
void launch_remove_mean(T* a, int count, int C, cudaStream_t st) {
  if (count <= 0) return;
  launch_pdl(remove_mean_kernel<T>, dim3(count), dim3(256), 0, st, a, C);
}

template <class Ts, class Td>
void launch_convert(const Ts* s, Td* d, size_t n, cudaStream_t st) {
  const int tpb = 256;
  unsigned nb = blocks_for(n, tpb);
  if (nb > 4096) nb = 4096;
  if (nb == 0) return;
  convert_kernel<Ts, Td><<<nb, tpb, 0, st>>>(s, d, n);
}

#define STC_INST_T(T)                                                                                     \
  template int launch_nso_residual<T>(const Geom&, CState<T>, const T*, CState<T>, State<T>, T, T,           \
                                      cudaStream_t, double*, const double*, RedScratch, void*, size_t);    \
  template int launch_nso_residual_colour<T>(const Geom&, CState<T>, const T*, CState<T>, State<T>, int,      \
                                             cudaStream_t, const double*, void*, size_t);                 \
  template int launch_scgs_colour<T>(const Geom&, State<T>, CState<T>, int, bool, cudaStream_t,           \
                                      const double*, void*);                                               \
  template void launch_absmax<T>(const T*, size_t, double*, int*, cudaStream_t);                          \
  template void launch_sumsq<T>(const T*, size_t, double*, cudaStream_t, RedScratch);                     \
  template void launch_remove_mean<T>(T*, int, int, cudaStream_t);
STC_INST_T(float)
STC_INST_T(double)

#define STC_INST_TT(Tf, Tc)                                                                                 \
  template void launch_restrict<Tf, Tc>(const Geom&, const Geom&, CState<Tf>, State<Tc>, State<Tc>,        \
                                        cudaStream_t);                                                     \
  template void launch_restrict_faces<Tf, Tc>(const Geom&, const Geom&, int, const Tf*, Tc*, cudaStream_t); \
  template void launch_prolong_correct<Tf, Tc>(const Geom&, const Geom&, State<Tf>, CState<Tc>, CState<Tc>, \
                                               cudaStream_t, const double*);                               \
  template void launch_convert<Tf, Tc>(const Tf*, Tc*, size_t, cudaStream_t);
STC_INST_TT(float, float)
STC_INST_TT(float, double)
STC_INST_TT(double, float)
STC_INST_TT(double, double)

}  // namespace stc
