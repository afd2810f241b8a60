// Internal definitions shared by the CUDA translation units of libstc.
//
// Discretisation (Sec. 3.1 of Pan & Manocha, "Efficient Optimal Control of
// Smoke using Spacetime Multigrid"): 2D staggered MAC grid, nx x ny cells of
// size h.  Centre fields (rho, p, pbar, mu) are [ny][nx] (i fastest).  A face
// field stores all x-faces [ny][nx+1] then all y-faces [ny+1][nx]; wall faces
// are stored and always hold 0 (closed box).  Time-dependent fields are slabs
// of one such array per timestep.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stc {

// Geometry and scalar parameters of one level, passed to kernels by value.
// dim = 2: the nx x ny grid above (nz = 1, Fxy = F).  dim = 3: the
// nx x ny x nz grid of grid3d.cuh (x-, y-, then z-faces; Fxy = Fx + Fy is the
// offset of the z-faces).
struct Geom {
  int nx, ny;        // cells
  int N;             // timesteps
  int Fx, F, C;      // x-face count, face count, cell count
  int dim, nz;       // 2 or 3; cells along z (1 in 2D)
  int Fy, Fxy;       // y-face count; x- plus y-face count
  int periodic;      // 3D only: 1 = every axis wraps (face slot n of an axis is unused)
  double h, ih;      // cell size and 1/h
  double dt, idt;    // timestep and 1/dt
  double a;          // K / r   (Eq. KKTAO row 1)
  double lm;         // Levenberg-Marquardt shift of the smoother's v blocks
  double omega;      // SCGS under-relaxation
  int self_adv;      // 1: Adv on (0 only for linear saddle tests)
  int cta_cells;     // 2D SCGS: colours of at most this many cells take the CTA-per-cell kernel (-1: by solve type)
  // the same scalars rounded to fp32 on the host (set_fp32_copies): fp32
  // kernels read these instead of converting fp64 scalars in every thread
  // (conversions from fp64 run at the much lower fp64 rate)
  float ihf, idtf, af, omegaf;
};

inline void set_fp32_copies(Geom& g) {
  g.ihf = (float)g.ih;
  g.idtf = (float)g.idt;
  g.af = (float)g.a;
  g.omegaf = (float)g.omega;
}

// geometry scalar in the arithmetic type: the fp32 copy or the fp64 value
template <class T> __host__ __device__ __forceinline__ T pick(double d, float f);
template <> __host__ __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __host__ __device__ __forceinline__ double pick<double>(double d, float) { return d; }

// NSO unknowns of one level: v (N+1)F, pbar (N+1)C, u N F, p N C  (p[i] = p_{i+1}).
template <class T>
struct State {
  T* v;
  T* pbar;
  T* u;
  T* p;
};

template <class T>
struct CState {
  const T* v;
  const T* pbar;
  const T* u;
  const T* p;
};

template <class T>
__host__ __device__ inline CState<T> cs(const State<T>& s) {
  return CState<T>{s.v, s.pbar, s.u, s.p};
}

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int xf(const Geom& g, int j, int i) { return j * (g.nx + 1) + i; }
__host__ __device__ inline int yf(const Geom& g, int j, int i) { return g.Fx + j * g.nx + i; }
__host__ __device__ inline int cidx(const Geom& g, int j, int i) { return j * g.nx + i; }

template <class T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// Deterministic fp64 sums.  Every block leaves its total in part[block]; the
// last block to take a ticket adds the partials in block order and adds the
// result to *out, then resets the ticket.  A sum therefore does not depend on
// the order in which the blocks ran (cross-block atomics did: a tie in a
// guard's comparison could then go either way between two runs).  cap: the
// entries of part (a launch must not have more blocks).
struct RedScratch {
  double* part;
  unsigned* ticket;
  unsigned cap;
};

// called by every thread of every block of the launch; v: this thread's share
__device__ inline void block_sum_ordered(double v, double* out, const RedScratch& rs) {
  __shared__ double wpart[32];
  __shared__ int last_s;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = v;
  __syncthreads();
  const int nw = (int)((blockDim.x + 31) >> 5);
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += wpart[k];
    rs.part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    __threadfence();
    last_s = atomicAdd(rs.ticket, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  double t = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x) t += __ldcg(rs.part + b);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += wpart[k];
    *out += s;
    *rs.ticket = 0;
  }
}

// Programmatic dependent launch: a kernel of the V-cycle chain may be launched
// while its predecessor is still finishing; it waits here, before touching any
// data, until the predecessor has completed and its writes are visible.  A
// no-op when the kernel was launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Row/column of e = threadIdx.x, threadIdx.x + blockDim.x, ... in a row-major
// range of rows of length P, advanced without a division per element.
struct RowWalk {
  int q, r, dq, dr, P;
  __device__ __forceinline__ RowWalk(int P_) : P(P_) {
    q = (int)threadIdx.x / P;
    r = (int)threadIdx.x - q * P;
    dq = (int)blockDim.x / P;
    dr = (int)blockDim.x - dq * P;
  }
  __device__ __forceinline__ void next() {
    q += dq;
    r += dr;
    if (r >= P) {
      r -= P;
      ++q;
    }
  }
};

// ---------------------------------------------------------------------------
// Self-advection Adv[v] = (curl v) x v  (Eq. NSA) and its Jacobian transpose.
// omega at node (j,i) = (vy(j,i)-vy(j,i-1))/h - (vx(j,i)-vx(j-1,i))/h, zero on
// wall nodes; Adv_x = -omega_bar * vbar_y, Adv_y = +omega_bar * vbar_x with
// omega_bar the mean of a face's two nodes and vbar the mean of the four
// surrounding transverse faces; Adv = 0 on wall faces.
// ---------------------------------------------------------------------------
// (T: element type of v; R: arithmetic type, T unless a caller asks otherwise)
template <class T, class R = T>
__device__ __forceinline__ R node_omega(const Geom& g, const T* v, int j, int i) {
  if (i <= 0 || i >= g.nx || j <= 0 || j >= g.ny) return R(0);
  R a = R(ld(v + yf(g, j, i))) - R(ld(v + yf(g, j, i - 1)));
  R b = R(ld(v + xf(g, j, i))) - R(ld(v + xf(g, j - 1, i)));
  return (a - b) * pick<R>(g.ih, g.ihf);
}

// transverse mean at an interior x-face (j,i)
template <class T, class R = T>
__device__ __forceinline__ R tv_x(const Geom& g, const T* v, int j, int i) {
  return R(0.25) * (R(ld(v + yf(g, j, i - 1))) + R(ld(v + yf(g, j, i))) + R(ld(v + yf(g, j + 1, i - 1))) +
                    R(ld(v + yf(g, j + 1, i))));
}

// transverse mean at an interior y-face (j,i)
template <class T, class R = T>
__device__ __forceinline__ R tv_y(const Geom& g, const T* v, int j, int i) {
  return R(0.25) * (R(ld(v + xf(g, j - 1, i))) + R(ld(v + xf(g, j - 1, i + 1))) + R(ld(v + xf(g, j, i))) +
                    R(ld(v + xf(g, j, i + 1))));
}

template <class T>
__device__ __forceinline__ T wbar_x(const Geom& g, const T* v, int j, int i) {
  return T(0.5) * (node_omega(g, v, j, i) + node_omega(g, v, j + 1, i));
}

template <class T>
__device__ __forceinline__ T wbar_y(const Geom& g, const T* v, int j, int i) {
  return T(0.5) * (node_omega(g, v, j, i) + node_omega(g, v, j, i + 1));
}

__device__ __forceinline__ bool xf_interior(const Geom& g, int j, int i) {
  return i >= 1 && i <= g.nx - 1 && j >= 0 && j < g.ny;
}
__device__ __forceinline__ bool yf_interior(const Geom& g, int j, int i) {
  return j >= 1 && j <= g.ny - 1 && i >= 0 && i < g.nx;
}

template <class T>
__device__ __forceinline__ T adv_x(const Geom& g, const T* v, int j, int i) {
  if (!xf_interior(g, j, i)) return T(0);
  return -wbar_x(g, v, j, i) * tv_x(g, v, j, i);
}

template <class T>
__device__ __forceinline__ T adv_y(const Geom& g, const T* v, int j, int i) {
  if (!yf_interior(g, j, i)) return T(0);
  return wbar_y(g, v, j, i) * tv_y(g, v, j, i);
}

// P_e = s_e * vbar_e * u_e on interior faces (s = -1 on x-faces, +1 on y-faces)
template <class T>
__device__ __forceinline__ T pe_x(const Geom& g, const T* v, const T* u, int j, int i) {
  if (!xf_interior(g, j, i)) return T(0);
  return -tv_x(g, v, j, i) * ld(u + xf(g, j, i));
}
template <class T>
__device__ __forceinline__ T pe_y(const Geom& g, const T* v, const T* u, int j, int i) {
  if (!yf_interior(g, j, i)) return T(0);
  return tv_y(g, v, j, i) * ld(u + yf(g, j, i));
}

// Q_n = 1/2 sum of P_e over the interior faces meeting at interior node n
template <class T>
__device__ __forceinline__ T node_q(const Geom& g, const T* v, const T* u, int j, int i) {
  if (i <= 0 || i >= g.nx || j <= 0 || j >= g.ny) return T(0);
  return T(0.5) * (pe_x(g, v, u, j - 1, i) + pe_x(g, v, u, j, i) + pe_y(g, v, u, j, i - 1) +
                   pe_y(g, v, u, j, i));
}

// (dAdv/dv)^T u at interior x-face (j,i): the node terms through omega plus the
// transverse-mean terms through vbar of the four y-faces averaging this face.
template <class T>
__device__ T jtu_x(const Geom& g, const T* v, const T* u, int j, int i) {
  T r = (node_q(g, v, u, j + 1, i) - node_q(g, v, u, j, i)) * pick<T>(g.ih, g.ihf);
  T s = T(0);
  if (yf_interior(g, j, i - 1)) s += wbar_y(g, v, j, i - 1) * ld(u + yf(g, j, i - 1));
  if (yf_interior(g, j, i)) s += wbar_y(g, v, j, i) * ld(u + yf(g, j, i));
  if (yf_interior(g, j + 1, i - 1)) s += wbar_y(g, v, j + 1, i - 1) * ld(u + yf(g, j + 1, i - 1));
  if (yf_interior(g, j + 1, i)) s += wbar_y(g, v, j + 1, i) * ld(u + yf(g, j + 1, i));
  return r + T(0.25) * s;
}

template <class T>
__device__ T jtu_y(const Geom& g, const T* v, const T* u, int j, int i) {
  T r = (node_q(g, v, u, j, i) - node_q(g, v, u, j, i + 1)) * pick<T>(g.ih, g.ihf);
  T s = T(0);
  if (xf_interior(g, j - 1, i)) s -= wbar_x(g, v, j - 1, i) * ld(u + xf(g, j - 1, i));
  if (xf_interior(g, j - 1, i + 1)) s -= wbar_x(g, v, j - 1, i + 1) * ld(u + xf(g, j - 1, i + 1));
  if (xf_interior(g, j, i)) s -= wbar_x(g, v, j, i) * ld(u + xf(g, j, i));
  if (xf_interior(g, j, i + 1)) s -= wbar_x(g, v, j, i + 1) * ld(u + xf(g, j, i + 1));
  return r + T(0.25) * s;
}

// gradient of a centre field at a face (zero on walls)
template <class T>
__device__ __forceinline__ T grad_x(const Geom& g, const T* p, int j, int i) {
  if (!xf_interior(g, j, i)) return T(0);
  return (ld(p + cidx(g, j, i)) - ld(p + cidx(g, j, i - 1))) * pick<T>(g.ih, g.ihf);
}
template <class T>
__device__ __forceinline__ T grad_y(const Geom& g, const T* p, int j, int i) {
  if (!yf_interior(g, j, i)) return T(0);
  return (ld(p + cidx(g, j, i)) - ld(p + cidx(g, j - 1, i))) * pick<T>(g.ih, g.ihf);
}

template <class T>
__device__ __forceinline__ T divergence(const Geom& g, const T* v, int j, int i) {
  return (ld(v + xf(g, j, i + 1)) - ld(v + xf(g, j, i)) + ld(v + yf(g, j + 1, i)) -
          ld(v + yf(g, j, i))) * pick<T>(g.ih, g.ihf);
}

// ---------------------------------------------------------------------------
// error flags written by kernels (host maps them to stc_status)
// ---------------------------------------------------------------------------
enum DevError : int {
  DEV_OK = 0,
  DEV_TAYLOR_KMAX = 1,   // Taylor series did not reach tolerance within kmax
  DEV_NONFINITE = 2,     // a non-finite value reached a norm
  DEV_BAD_LAUNCH = 4,    // launch shape inconsistent with the data (bounds guard)
  DEV_BARRIER_TIMEOUT = 8,   // a grid-wide barrier waited past its iteration limit
};

}  // namespace stc
