// Passive advection by the truncated Taylor exponential (Sec. 3.1, Eq. Adv)
// and the backward adjoint sweep of the AO fixed point (Eq. KKTPO, Alg. 1).
//
// Both sweeps are sequential in time and, inside a step, sequential in the
// Taylor order; they run as ONE launch of an 8-CTA thread-block cluster per
// problem.  Each CTA owns a slab of grid rows; the term fields live in shared
// memory with a 2-row halo that is copied from the neighbouring CTAs through
// distributed shared memory after every cluster barrier (QUICK needs two
// upwind cells).  The truncation order of a step is decided from the
// cluster-wide max |t_k|, so all CTAs take the same decision.
#include <cooperative_groups.h>

#include <mutex>
#include <vector>

#include "../../include/stc.h"
#include "stc_internal.cuh"
#include "stc_kernels.h"

namespace cg = cooperative_groups;

namespace stc {

struct Slab {
  int r0, r1, rpc;  // owned rows [r0, r1), rows per CTA
};

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// QUICK (Leonard) coefficients of one face between cells lo and hi: the
// weights of (lo, hi, lo-1, hi+1) in the face value, the far cells clamped at
// the walls.  v > 0: upwind lo; v < 0: upwind hi; v = 0: the mean of both
// one-sided stencils (the subgradient used for d/dv at v = 0).
template <class T>
__device__ __forceinline__ void quick_coef(T v, T c[4]) {
  const bool pos = v > T(0), neg = v < T(0);
  c[0] = pos ? T(0.75) : (neg ? T(0.375) : T(0.5625));
  c[1] = pos ? T(0.375) : (neg ? T(0.75) : T(0.5625));
  c[2] = pos ? T(-0.125) : (neg ? T(0) : T(-0.0625));
  c[3] = pos ? T(0) : (neg ? T(-0.125) : T(-0.0625));
}

// row jj (clamped to the grid) of a slab buffer with a 2-row halo
template <class T>
__device__ __forceinline__ const T* buf_row(const Geom& g, const Slab& s, const T* b, int jj) {
  jj = clampi(jj, 0, g.ny - 1);
  return b + (jj - s.r0 + 2) * g.nx;
}


// Face arrays of a slab: x-faces of the owned rows [r0, r1) (all columns),
// y-faces of rows [r0 - 1, r0 + rpc + 1] (row index offset by 1).
__device__ __forceinline__ int nxf(const Geom& g, const Slab& s) { return s.rpc * (g.nx + 1); }
__device__ __forceinline__ int nyf(const Geom& g, const Slab& s) { return (s.rpc + 3) * g.nx; }

template <class T>
__device__ void load_velocity(const Geom& g, const Slab& s, const T* vel, T* vx, T* vy) {
  const int nx = g.nx;
  RowWalk wx(nx + 1);
  for (int e = threadIdx.x; e < nxf(g, s); e += blockDim.x, wx.next()) {
    const int j = s.r0 + wx.q;
    vx[e] = (j < s.r1) ? vel[(size_t)s.r0 * (nx + 1) + e] : T(0);
  }
  RowWalk wy(nx);
  for (int e = threadIdx.x; e < nyf(g, s); e += blockDim.x, wy.next()) {
    const int jf = s.r0 - 1 + wy.q, i = wy.r;
    vy[e] = (jf >= 0 && jf <= g.ny && s.r1 > s.r0) ? vel[g.Fx + (size_t)jf * nx + i] : T(0);
  }
}

// fluxes F_f = v_f * QUICK(t)_f on the faces the owned cells need
template <class T>
__device__ void face_fluxes(const Geom& g, const Slab& s, const T* t, const T* vx, const T* vy, T* Fx, T* Fy) {
  const int nx = g.nx;
  const int nown = s.r1 - s.r0;
  RowWalk wx(nx + 1);
  for (int e = threadIdx.x; e < nown * (nx + 1); e += blockDim.x, wx.next()) {
    const int j = s.r0 + wx.q, i = wx.r;
    T F = T(0);
    const T v = vx[e];
    if (i >= 1 && i <= nx - 1 && v != T(0)) {
      T c[4];
      quick_coef(v, c);
      const T* row = buf_row(g, s, t, j);
      F = v * (c[0] * row[i - 1] + c[1] * row[i] + c[2] * row[max(i - 2, 0)] + c[3] * row[min(i + 1, nx - 1)]);
    }
    Fx[e] = F;
  }
  // y-faces r0 .. r1 (local rows 1 .. nown + 1)
  RowWalk wy(nx);
  for (int e = threadIdx.x; e < (nown + 1) * nx; e += blockDim.x, wy.next()) {
    const int jf = s.r0 + wy.q, i = wy.r;
    const int le = e + nx;
    T F = T(0);
    const T v = vy[le];
    if (jf >= 1 && jf <= g.ny - 1 && v != T(0)) {
      T c[4];
      quick_coef(v, c);
      F = v * (c[0] * buf_row(g, s, t, jf - 1)[i] + c[1] * buf_row(g, s, t, jf)[i] +
               c[2] * buf_row(g, s, t, jf - 2)[i] + c[3] * buf_row(g, s, t, jf + 1)[i]);
    }
    Fy[le] = F;
  }
}

// (A t)_c = -(1/h) sum_a (F_{c+1/2} - F_{c-1/2}) at owned cell e (slab-local index)
template <class T>
__device__ __forceinline__ T flux_divergence(const Geom& g, const T* Fx, const T* Fy, int lj, int i) {
  const int nx = g.nx;
  const int xr = lj * (nx + 1) + i;
  const int yr = (lj + 1) * nx + i;
  return -pick<T>(g.ih, g.ihf) * (Fx[xr + 1] - Fx[xr] + Fy[yr + nx] - Fy[yr]);
}

// E_f = v_f (w_hi - w_lo) / h on the faces within two cells of the owned rows
template <class T>
__device__ void face_differences(const Geom& g, const Slab& s, const T* w, const T* vx, const T* vy, T* Ex, T* Ey,
                                 T* Gx, T* Gy) {
  const int nx = g.nx;
  const int nown = s.r1 - s.r0;
  const T ih = pick<T>(g.ih, g.ihf);
  RowWalk wx(nx + 1);
  for (int e = threadIdx.x; e < nown * (nx + 1); e += blockDim.x, wx.next()) {
    const int j = s.r0 + wx.q, i = wx.r;
    T d = T(0);
    if (i >= 1 && i <= nx - 1) {
      const T* row = buf_row(g, s, w, j);
      d = (row[i] - row[i - 1]) * ih;
    }
    Gx[e] = d;
    Ex[e] = vx[e] * d;
  }
  RowWalk wy(nx);
  for (int e = threadIdx.x; e < nyf(g, s); e += blockDim.x, wy.next()) {
    const int jf = s.r0 - 1 + wy.q, i = wy.r;
    T d = T(0);
    if (jf >= 1 && jf <= g.ny - 1 && jf <= s.r1 + 1 && s.r1 > s.r0)
      d = (buf_row(g, s, w, jf)[i] - buf_row(g, s, w, jf - 1)[i]) * ih;
    Gy[e] = d;
    Ey[e] = vy[e] * d;
  }
}

// (A^T w)_c = sum over faces f whose QUICK stencil holds c of coef(f, c) E_f;
// along one axis of n cells, cell i is hi of face i, lo of face i+1, lo-1 of
// face i+2 and hi+1 of face i-1, plus the wall-clamped extras of faces 1 and n-1.
template <class T>
__device__ __forceinline__ T gather_axis(const T* v, const T* E, int stride, int i, int n) {
  T acc = T(0), c[4];
  if (i >= 1) { quick_coef(v[i * stride], c); acc += c[1] * E[i * stride]; }
  if (i + 1 <= n - 1) { quick_coef(v[(i + 1) * stride], c); acc += c[0] * E[(i + 1) * stride]; }
  if (i + 2 <= n - 1) { quick_coef(v[(i + 2) * stride], c); acc += c[2] * E[(i + 2) * stride]; }
  if (i - 1 >= 1) { quick_coef(v[(i - 1) * stride], c); acc += c[3] * E[(i - 1) * stride]; }
  if (i == 0 && n >= 2) { quick_coef(v[stride], c); acc += c[2] * E[stride]; }
  if (i == n - 1 && n >= 2) { quick_coef(v[(n - 1) * stride], c); acc += c[3] * E[(n - 1) * stride]; }
  return acc;
}

template <class T>
__device__ __forceinline__ T apply_AT_cell(const Geom& g, const Slab& s, const T* vx, const T* vy, const T* Ex,
                                           const T* Ey, int lj, int i) {
  const int nx = g.nx;
  const int j = s.r0 + lj;
  // x: faces of row j, index i' in [0, nx]
  const T ax = gather_axis(vx + lj * (nx + 1), Ex + lj * (nx + 1), 1, i, nx);
  // y: faces of column i, face row jf at local row jf - r0 + 1; pass pointers shifted so that
  // index jf addresses face row jf
  const T* vyc = vy + (1 - s.r0) * nx + i;
  const T* Eyc = Ey + (1 - s.r0) * nx + i;
  const T ay = gather_axis(vyc, Eyc, nx, j, g.ny);
  return ax + ay;
}

// Asynchronous global -> shared copies of single elements (cp.async, sm_80+);
// the issuing thread waits for its own copies with cp_async_wait_all, a block
// barrier after that makes them visible to the block.
template <int B>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (B == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Start copying rows [max(r0-2, 0), min(r1+1, ny-1)] of a cell field P (global)
// into Ps; returns the first staged row.  These are all the rows the QUICK
// stencils of the owned faces read (accumulate_grad).
template <class T>
__device__ int stage_term_rows(const Geom& g, const Slab& s, const T* P, T* Ps) {
  const int rlo = max(s.r0 - 2, 0), rhi = min(s.r1 + 1, g.ny - 1);
  const int n = s.r1 > s.r0 ? (rhi - rlo + 1) * g.nx : 0;
  const T* src = P + (size_t)rlo * g.nx;
  for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async_elem<sizeof(T)>(Ps + e, src + e);
  cp_async_commit();
  return rlo;
}

// B(P)^T at the owned faces: QUICK(P)_f * (w_hi - w_lo)/h, P staged in shared
// memory (rows from rlo, see stage_term_rows)
template <class T>
__device__ void accumulate_grad(const Geom& g, const Slab& s, const T* Ps, int rlo, const T* vx, const T* vy,
                                const T* Gx, const T* Gy, T* gxs, T* gys) {
  const int nx = g.nx;
  const int nown = s.r1 - s.r0;
  RowWalk wx(nx + 1);
  for (int e = threadIdx.x; e < nown * (nx + 1); e += blockDim.x, wx.next()) {
    const int j = s.r0 + wx.q, i = wx.r;
    if (i >= 1 && i <= nx - 1) {
      T c[4];
      quick_coef(vx[e], c);
      const T* row = Ps + (size_t)(j - rlo) * nx;
      gxs[e] += (c[0] * row[i - 1] + c[1] * row[i] + c[2] * row[max(i - 2, 0)] + c[3] * row[min(i + 1, nx - 1)]) *
                Gx[e];
    }
  }
  RowWalk wy(nx);
  for (int e = threadIdx.x; e < nown * nx; e += blockDim.x, wy.next()) {
    const int jf = s.r0 + wy.q, i = wy.r;
    if (jf >= 1 && jf <= g.ny - 1) {
      T c[4];
      const int le = e + nx;
      quick_coef(vy[le], c);
      gys[e] += (c[0] * Ps[(size_t)(jf - 1 - rlo) * nx + i] + c[1] * Ps[(size_t)(jf - rlo) * nx + i] +
                 c[2] * Ps[(size_t)(max(jf - 2, 0) - rlo) * nx + i] +
                 c[3] * Ps[(size_t)(min(jf + 1, g.ny - 1) - rlo) * nx + i]) *
                Gy[le];
    }
  }
}

// Push this CTA's rows that other CTAs need as halo (rows within 2 of its slab
// edges) into their copy of buffer `b` (same shared-memory offset in every CTA)
// with remote stores; the next cluster barrier publishes them.  No CTA reads
// remote shared memory on the critical path.
template <class T>
__device__ void halo_push(cg::cluster_group& cl, const Geom& g, const Slab& s, T* b, int rank) {
  const int nx = g.nx;
  if (s.r1 <= s.r0) return;
  for (int e = threadIdx.x; e < 4 * nx; e += blockDim.x) {
    const int q = e / nx, i = e - q * nx;
    const int jj = (q < 2) ? s.r0 + q : s.r1 - 4 + q;   // r0, r0+1, r1-2, r1-1
    if (jj < s.r0 || jj >= s.r1) continue;
    if (q >= 2 && jj < s.r0 + 2) continue;               // already pushed as r0 / r0+1
    const T val = b[(jj - s.r0 + 2) * nx + i];
    int last = -1;
    for (int d = -2; d <= 2; ++d) {
      const int row = jj + d;
      if (d == 0 || row < 0 || row >= g.ny) continue;
      const int owner = row / s.rpc;
      if (owner == rank || owner == last) continue;
      last = owner;
      const int r0o = owner * s.rpc;
      const int r1o = min(g.ny, r0o + s.rpc);
      if ((jj >= r0o - 2 && jj < r0o) || (jj >= r1o && jj < r1o + 2)) {
        T* rb = cl.map_shared_rank(b, owner);
        rb[(jj - r0o + 2) * nx + i] = val;
      }
    }
  }
}

// Shared-memory layout of both sweeps (element counts of T arrays, then the
// fp64 cluster-max slots at a 16-byte-aligned byte offset).
template <class T>
struct AdvLayout {
  size_t buf, fx, fy, gx, gy, ps;
  size_t cm_off;
  size_t total;
};

template <class T>
__host__ __device__ inline AdvLayout<T> adv_layout(const Geom& g, bool adjoint, int ncta) {
  const int rpc = (g.ny + ncta - 1) / ncta;
  AdvLayout<T> L;
  L.buf = (size_t)(rpc + 4) * g.nx;
  L.fx = (size_t)rpc * (g.nx + 1);
  L.fy = (size_t)(rpc + 3) * g.nx;
  L.gx = adjoint ? L.fx : 0;
  L.gy = adjoint ? L.fy : 0;
  L.ps = adjoint ? (size_t)(rpc + 4) * g.nx : 0;   // staged rows of a series term
  // tb0, tb1, vx, vy, Fx (E), Fy (E), [Gx, Gy, gxs, gys, Ps]
  const size_t n = 2 * L.buf + 2 * L.fx + 2 * L.fy + (adjoint ? 2 * L.fx + 2 * L.fy + L.ps : 0);
  L.cm_off = (n * sizeof(T) + 15) / 16 * 16;
  L.total = L.cm_off + 2 * kMaxClusterCTAs * sizeof(double);
  return L;
}

__device__ __forceinline__ Slab make_slab(const Geom& g, int rank, int ncta) {
  Slab s;
  s.rpc = (g.ny + ncta - 1) / ncta;
  s.r0 = rank * s.rpc;
  if (s.r0 > g.ny) s.r0 = g.ny;
  s.r1 = s.r0 + s.rpc;
  if (s.r1 > g.ny) s.r1 = g.ny;
  return s;
}

// Block-wide max of non-negative values.  A max is exact in any precision, so
// the series' stopping test reduces in the state type (fp64 arithmetic runs at
// a small fraction of the fp32 rate) and compares with its fp64 threshold
// only at the end: the decision is the same as reducing in fp64.
template <class T>
__device__ __forceinline__ T block_max(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T m = T(0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  return m;
}

// dt / k for k = 1..kmax, formed once per launch in fp64 and rounded to T
// (the per-term quotient would otherwise be an fp64 division in every thread)
template <class T>
__device__ __forceinline__ void fill_dt_over_k(const Geom& g, int kmax, T* tab) {
  for (int k = (int)threadIdx.x + 1; k <= kmax; k += blockDim.x) tab[k] = T(g.dt / k);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// forward sweep: rho_{s+1} = sum_{k<=K} (dt^k/k!) A(v_s)^k rho_s, K the first
// order with max|t_k| < thresh (the small term included).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kAdvThreads, 1)
taylor_forward_kernel(Geom g, const T* __restrict__ vel, T* rho, int* Ks, double thresh, int kmax, int* err) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int ncta = (int)cl.num_blocks();
  const Slab s = make_slab(g, rank, ncta);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const AdvLayout<T> L = adv_layout<T>(g, false, ncta);
  T* tb0 = reinterpret_cast<T*>(smem_raw);
  T* tb1 = tb0 + L.buf;
  T* vx = tb1 + L.buf;
  T* vy = vx + L.fx;
  T* Fx = vy + L.fy;
  T* Fy = Fx + L.fx;
  T* cmax = reinterpret_cast<T*>(smem_raw + L.cm_off);
  __shared__ T red[32];
  __shared__ T dtk[kTaylorKmaxLimit + 1];
  fill_dt_over_k(g, kmax, dtk);
  const int nown = (s.r1 - s.r0) * g.nx;

  T acc[kAdvMaxCellsPerThread], cmp[kAdvMaxCellsPerThread];
  int clj[kAdvMaxCellsPerThread], cii[kAdvMaxCellsPerThread];   // slab row / column of each owned cell
#pragma unroll
  for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    acc[q] = (e < nown) ? rho[(size_t)s.r0 * g.nx + e] : T(0);
    cmp[q] = T(0);
    clj[q] = e / g.nx;
    cii[q] = e - clj[q] * g.nx;
  }
  int kfail = 0;
  for (int st = 0; st < g.N; ++st) {
    // t_0 = rho_st into tb0 own rows, its halo pushed; velocity of step st
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) tb0[2 * g.nx + e] = acc[q];
    }
    load_velocity(g, s, vel + (size_t)st * g.F, vx, vy);
    __syncthreads();
    halo_push(cl, g, s, tb0, rank);
    cl.sync();
    T* cur = tb0;
    T* nxt = tb1;
    int K = kmax;
    bool done = false;
    for (int k = 1; k <= kmax; ++k) {
      face_fluxes(g, s, cur, vx, vy, Fx, Fy);
      __syncthreads();
      const T ck = dtk[k];
      T lmax = T(0);
#pragma unroll
      for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < nown) {
          const T t = ck * flux_divergence(g, Fx, Fy, clj[q], cii[q]);
          nxt[2 * g.nx + e] = t;
          // two-sum accumulation of the series
          const T sum = acc[q] + t;
          const T bb = sum - acc[q];
          cmp[q] += (acc[q] - (sum - bb)) + (t - bb);
          acc[q] = sum;
          lmax = fmax(lmax, fabs(t));
        }
      }
      const T bm = block_max(lmax, red);   // also orders the nxt writes before the push
      halo_push(cl, g, s, nxt, rank);
      if ((int)threadIdx.x < ncta)
        *cl.map_shared_rank(cmax + (k & 1) * kMaxClusterCTAs + rank, (int)threadIdx.x) = bm;
      cl.sync();
      T gm = T(0);
#pragma unroll
      for (int r = 0; r < ncta; ++r) gm = fmax(gm, cmax[(k & 1) * kMaxClusterCTAs + r]);
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
      if ((double)gm < thresh) {
        K = k;
        done = true;
        break;
      }
    }
    if (!done) kfail = 1;
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) {
        acc[q] += cmp[q];
        cmp[q] = T(0);
        rho[(size_t)(st + 1) * g.C + (size_t)s.r0 * g.nx + e] = acc[q];
      }
    }
    if (rank == 0 && threadIdx.x == 0) Ks[st] = K;
  }
  if (kfail && threadIdx.x == 0) atomicOr(err, DEV_TAYLOR_KMAX);
  cl.sync();
}

// ---------------------------------------------------------------------------
// backward sweep.  For s = N-1 .. 1 with mu_s known, with c_m = dt^m / m!:
//   Taylor terms t_m = c_m A^m rho_s (m < K_s) -> global scratch
//   Horner  w_{K-1} = c_K mu, w_{m-1} = c_m mu + A^T w_m
//   grad    = sum_m B(A^m rho_s)^T w_m  = (dA[rho_s, v_s]/dv_s)^T mu_s
//   T^T mu  = w_{-1};  mu_{s-1} = T^T mu_s - m_s
// evaluated in the scaled variables w'_m = w_m / c_m, so that every stored
// quantity stays bounded like the series terms (the raw powers A^m rho grow
// like ||A||^m and overflowed fp32 at m ~ 17 on strong flows):
//   w'_{K-1} = (dt/K) mu,  w'_{m-1} = (dt/m)(mu + A^T w'_m),
//   grad = sum_m B(t_m)^T w'_m,  T^T mu = mu + A^T w'_0.
// B(x)^T w at a face = QUICK(x)_face * (w_hi - w_lo) / h.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kAdvThreads, 1)
taylor_adjoint_kernel(Geom g, const T* __restrict__ vel, const T* __restrict__ rho, const int* __restrict__ Ks,
                      const double* __restrict__ mterm, T* mu, const T* __restrict__ base, T alpha, T beta,
                      T* out, T* powers, int kmax, int s_end, T* mu_m1, int* err) {
  __shared__ T dtk[kTaylorKmaxLimit + 1];
  fill_dt_over_k(g, kmax, dtk);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int ncta = (int)cl.num_blocks();
  const Slab s = make_slab(g, rank, ncta);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const AdvLayout<T> L = adv_layout<T>(g, true, ncta);
  T* tb0 = reinterpret_cast<T*>(smem_raw);
  T* tb1 = tb0 + L.buf;
  T* vx = tb1 + L.buf;
  T* vy = vx + L.fx;
  T* Ex = vy + L.fy;
  T* Ey = Ex + L.fx;
  T* Gx = Ey + L.fy;
  T* Gy = Gx + L.fx;
  T* gxs = Gy + L.fy;
  T* gys = gxs + L.fx;
  T* Ps = gys + L.fy;
  const int nx = g.nx;
  const int nown = (s.r1 - s.r0) * nx;
  const int ngx = (s.r1 - s.r0) * (nx + 1);
  const int ngy = (s.r1 - s.r0) * nx;

  T m[kAdvMaxCellsPerThread];
  int clj[kAdvMaxCellsPerThread], cii[kAdvMaxCellsPerThread];   // slab row / column of each owned cell
#pragma unroll
  for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    m[q] = (e < nown) ? T(-mterm[(size_t)g.N * g.C + (size_t)s.r0 * nx + e]) : T(0);
    clj[q] = e / nx;
    cii[q] = e - clj[q] * nx;
  }
  for (int st = g.N - 1; st >= s_end; --st) {
    // every CTA has finished the previous step (halo reads of the term
    // buffers, reads of the global powers) before they are overwritten
    cl.sync();
    const size_t cbase = (size_t)st * g.C + (size_t)s.r0 * nx;
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) mu[cbase + e] = m[q];
    }
    int K = Ks[st];
    if (K < 1 || K > kmax) {
      // an order the powers buffer cannot hold: flagged, and the sweep
      // continues with the clamped order (its output is then not the adjoint)
      if (err && rank == 0 && threadIdx.x == 0) atomicOr(err, DEV_TAYLOR_KMAX);
      K = K < 1 ? 1 : kmax;
    }
    const T* rs = rho + (size_t)st * g.C;
    load_velocity(g, s, vel + (size_t)st * g.F, vx, vy);
    // powers P_1 .. P_{K-1}
    for (int e = threadIdx.x; e < nown; e += blockDim.x) tb0[2 * nx + e] = rs[(size_t)s.r0 * nx + e];
    __syncthreads();
    halo_push(cl, g, s, tb0, rank);
    T* cur = tb0;
    T* nxt = tb1;
    for (int k = 1; k < K; ++k) {
      cl.sync();
      face_fluxes(g, s, cur, vx, vy, Ex, Ey);
      __syncthreads();
      const T ck = dtk[k];
      RowWalk wc(nx);
      for (int e = threadIdx.x; e < nown; e += blockDim.x, wc.next()) {
        const T t = ck * flux_divergence(g, Ex, Ey, wc.q, wc.r);
        nxt[2 * nx + e] = t;
        powers[(size_t)k * g.C + (size_t)s.r0 * nx + e] = t;
      }
      __syncthreads();
      halo_push(cl, g, s, nxt, rank);
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    for (int e = threadIdx.x; e < ngx; e += blockDim.x) gxs[e] = T(0);
    for (int e = threadIdx.x; e < ngy; e += blockDim.x) gys[e] = T(0);
    cl.sync();  // terms visible to the cluster; everyone done with tb buffers
    cur = tb0;
    nxt = tb1;
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) cur[2 * nx + e] = dtk[K] * m[q];   // w'_{K-1}
    }
    __syncthreads();
    halo_push(cl, g, s, cur, rank);
    for (int mm = K - 1; mm >= 0; --mm) {
      cl.sync();
      // the rows of t_m this CTA's stencils read, copied while E and G are formed
      const int rlo = stage_term_rows(g, s, (mm == 0) ? rs : powers + (size_t)mm * g.C, Ps);
      face_differences(g, s, cur, vx, vy, Ex, Ey, Gx, Gy);
      cp_async_wait_all();
      __syncthreads();
      // grad += B(t_m)^T w'_m on own faces
      accumulate_grad(g, s, Ps, rlo, vx, vy, Gx, Gy, gxs, gys);
      // w'_{m-1} = (dt/m)(mu + A^T w'_m); for m = 0 the factor is 1 (T^T mu)
      const T fac = (mm == 0) ? T(1) : dtk[mm];
#pragma unroll
      for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < nown) nxt[2 * nx + e] = fac * (m[q] + apply_AT_cell(g, s, vx, vy, Ex, Ey, clj[q], cii[q]));
      }
      __syncthreads();
      halo_push(cl, g, s, nxt, rank);
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    __syncthreads();
    // outputs for step st; mu_{st-1} = T^T mu_st - m_st
    const size_t fb = (size_t)st * g.F;
    for (int e = threadIdx.x; e < ngx; e += blockDim.x) {
      const size_t f = (size_t)s.r0 * (nx + 1) + e;
      T b = base ? base[fb + f] : T(0);
      out[fb + f] = alpha * b + beta * gxs[e];
    }
    for (int e = threadIdx.x; e < ngy; e += blockDim.x) {
      const size_t f = (size_t)g.Fx + (size_t)s.r0 * nx + e;
      T b = base ? base[fb + f] : T(0);
      out[fb + f] = alpha * b + beta * gys[e];
    }
    if (s.r1 == g.ny && s.r1 > s.r0) {
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const size_t f = (size_t)g.Fx + (size_t)g.ny * nx + i;
        T b = base ? base[fb + f] : T(0);
        out[fb + f] = alpha * b;
      }
    }
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) m[q] = cur[2 * nx + e] - T(mterm[cbase + e]);
    }
  }
  // mu_0, or with s_end = 0 the adjoint density of step 0 (T_0^T mu_0 - m_0)
  T* mu_out = s_end == 0 ? mu_m1 : mu;
  if (mu_out) {
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) mu_out[(size_t)s.r0 * nx + e] = m[q];
    }
  }
  cl.sync();
}

// ---------------------------------------------------------------------------
// keyframe metric: m = c * sum_l G_l^T G_l (rho - rho*), separable Gaussian
// filters (sigma_l = sigma0 2^l cells, taps to ceil(3 sigma), normalised,
// clamp-to-edge).  G^T is evaluated as a gather of the clamped-tap matrix;
// its first and last columns collect whole tails of the taps, read from a
// prefix sum of the weights.  Arithmetic in the state type Tc (fp32 in the
// fp32 policy: the metric term feeds the fp32 adjoint sweep); the weights are
// formed in fp64 and the result is accumulated into the fp64 metric slab.
// ---------------------------------------------------------------------------
// One separable pass for every level at once: level l = blockIdx.y filters
// in + l in_stride into out + l out_stride with sigma_l = sigma0 2^l.
template <class Tc, class To>
__global__ void blur_kernel(int nx, int ny, int axis, int transpose, double sigma0, const Tc* __restrict__ in,
                            size_t in_stride, To* out, size_t out_stride, double scale) {
  extern __shared__ double wsm[];
  const double sigma = sigma0 * (double)(1 << blockIdx.y);
  in += (size_t)blockIdx.y * in_stride;
  out += (size_t)blockIdx.y * out_stride;
  const int R = (int)ceil(3.0 * sigma);
  const int nt = 2 * R + 1;
  double* wd = wsm;              // raw weights, then their prefix sums (fp64)
  Tc* w = reinterpret_cast<Tc*>(wsm + nt);        // normalised weights
  Tc* cw = w + nt;                                 // cw[k] = w[0] + ... + w[k]
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double d = t - R;
    wd[t] = exp(-d * d / (2.0 * sigma * sigma));
  }
  __syncthreads();
  // inclusive prefix sums of the raw weights: a parallel scan when the taps
  // fit the block, else one thread
  const double raw = threadIdx.x < nt ? wd[threadIdx.x] : 0.0;
  if (nt <= (int)blockDim.x) {
    for (int off = 1; off < nt; off <<= 1) {
      const double add = (threadIdx.x < nt && (int)threadIdx.x >= off) ? wd[threadIdx.x - off] : 0.0;
      __syncthreads();
      if (threadIdx.x < nt) wd[threadIdx.x] += add;
      __syncthreads();
    }
  } else {
    if (threadIdx.x == 0)
      for (int t = 1; t < nt; ++t) wd[t] += wd[t - 1];
    __syncthreads();
  }
  const double inv = 1.0 / wd[nt - 1];
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double rt = nt <= (int)blockDim.x ? raw : (t > 0 ? wd[t] - wd[t - 1] : wd[0]);
    w[t] = Tc(rt * inv);
    cw[t] = Tc(wd[t] * inv);
  }
  __syncthreads();
  const int n = axis == 0 ? nx : ny;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nx * ny; e += gridDim.x * blockDim.x) {
    const int j = e / nx, i = e % nx;
    const int a = axis == 0 ? i : j;
    auto at = [&](int b) { return axis == 0 ? in[j * nx + b] : in[b * nx + i]; };
    Tc acc = Tc(0);
    if (!transpose) {
      for (int t = -R; t <= R; ++t) acc += w[t + R] * at(clampi(a + t, 0, n - 1));
    } else {
      // (G^T y)_a = sum_b G[b,a] y_b, G[b,a] = sum_t w_t [clamp(b+t) == a]
      const int lo = a - R < 0 ? 0 : a - R, hi = a + R > n - 1 ? n - 1 : a + R;
      if (n == 1) {
        acc = at(0);
      } else if (a == 0) {            // taps t <= -b clamp onto column 0
        for (int b = lo; b <= hi; ++b) acc += cw[R - b] * at(b);
      } else if (a == n - 1) {        // taps t >= n-1-b clamp onto column n-1
        for (int b = lo; b <= hi; ++b) {
          const int k0 = n - 2 - b + R;      // prefix index just below the tail
          acc += (cw[2 * R] - (k0 >= 0 ? cw[k0] : Tc(0))) * at(b);
        }
      } else {
        for (int b = lo; b <= hi; ++b) acc += w[a - b + R] * at(b);
      }
    }
    out[e] = To(acc * Tc(scale));
  }
}

// out = sum over the levels, in level order from zero, of the per-level terms
template <class Tc>
__global__ void level_sum_kernel(const Tc* __restrict__ v, int levels, int C, double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < levels; ++l) acc += (double)v[(size_t)l * C + e];
    out[e] = acc;
  }
}

template <class T, class Tc>
__global__ void metric_diff_kernel(const T* __restrict__ rho, const double* __restrict__ star, Tc* d, int C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C; e += gridDim.x * blockDim.x)
    d[e] = Tc((double)rho[e] - star[e]);
}

template <class Tc>
__global__ void scale_kernel(const Tc* __restrict__ in, double* out, double c, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) out[e] = c * (double)in[e];
}

size_t metric_tmp1_doubles(size_t C, int levels) { return 2 * C * (size_t)(levels > 1 ? levels : 1); }

// tmp0: C doubles, tmp1: metric_tmp1_doubles (used as arrays of the state
// type: per level, G_x d and G_y^T G_y G_x d, then c G_x^T of that).  Each
// pass runs every level in one launch; the levels are summed in level order
// at the end, as the per-level accumulation did.
template <class T>
void launch_metric(const Geom& g, const T* rho_s, const double* star, double c, int levels, double sigma0,
                   double* out, double* tmp0, double* tmp1, cudaStream_t st) {
  if (g.dim == 3) return launch_metric3<T>(g, rho_s, star, c, levels, sigma0, out, tmp0, tmp1, st);
  const int C = g.C;
  const int tpb = 256;
  const unsigned nb = (unsigned)((C + tpb - 1) / tpb);
  T* d0 = reinterpret_cast<T*>(tmp0);
  T* d1 = reinterpret_cast<T*>(tmp1);            // [levels][C]
  T* d2 = d1 + (size_t)levels * C;               // [levels][C]
  metric_diff_kernel<T, T><<<nb, tpb, 0, st>>>(rho_s, star, d0, C);
  if (levels <= 0) {
    scale_kernel<T><<<nb, tpb, 0, st>>>(d0, out, c, C);   // C_i = c_i I
    return;
  }
  const int R = (int)ceil(3.0 * sigma0 * (double)(1 << (levels - 1)));   // the widest level's taps
  const size_t sm = sizeof(double) * 3 * (2 * R + 1);
  const dim3 grid(nb, levels);
  const size_t Cs = (size_t)C;
  blur_kernel<T, T><<<grid, tpb, sm, st>>>(g.nx, g.ny, 0, 0, sigma0, d0, 0, d1, Cs, 1.0);   // G_x
  blur_kernel<T, T><<<grid, tpb, sm, st>>>(g.nx, g.ny, 1, 0, sigma0, d1, Cs, d2, Cs, 1.0);  // G_y
  blur_kernel<T, T><<<grid, tpb, sm, st>>>(g.nx, g.ny, 1, 1, sigma0, d2, Cs, d1, Cs, 1.0);  // G_y^T
  blur_kernel<T, T><<<grid, tpb, sm, st>>>(g.nx, g.ny, 0, 1, sigma0, d1, Cs, d2, Cs, c);    // c G_x^T
  level_sum_kernel<T><<<nb, tpb, 0, st>>>(d2, levels, C, out);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
bool advect_supported(const Geom& g) {
  const int ncta = advect_cluster_ctas();
  const int rpc = (g.ny + ncta - 1) / ncta;
  return g.nx >= 2 && g.ny >= 2 && rpc * g.nx <= kAdvThreads * kAdvMaxCellsPerThread;
}
size_t advect_smem_forward(const Geom& g, size_t tsize) {
  const int n = advect_cluster_ctas();
  return tsize == 4 ? adv_layout<float>(g, false, n).total : adv_layout<double>(g, false, n).total;
}
size_t advect_smem_adjoint(const Geom& g, size_t tsize) {
  const int n = advect_cluster_ctas();
  return tsize == 4 ? adv_layout<float>(g, true, n).total : adv_layout<double>(g, true, n).total;
}

// The dynamic shared-memory cap of a kernel is raised once, to the opt-in
// maximum, rather than to each launch's size: problems of different sizes
// launched from several host threads would otherwise race on the attribute.
static cudaError_t allow_max_smem(const void* kernel) {
  static std::mutex mu;
  static std::vector<const void*> done;
  std::lock_guard<std::mutex> lock(mu);
  for (const void* k : done)
    if (k == kernel) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, kernel);
  // the cap covers dynamic memory only: opt-in total minus the static arrays
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err == cudaSuccess) done.push_back(kernel);
  return err;
}

template <class T>
__global__ void __launch_bounds__(kAdvThreads, 1)
taylor_adjoint_kernel(Geom g, const T* __restrict__ vel, const T* __restrict__ rho, const int* __restrict__ Ks,
                      const double* __restrict__ mterm, T* mu, const T* __restrict__ base, T alpha, T beta,
                      T* out, T* powers, int kmax, int s_end, T* mu_m1, int* err);

// A 16-CTA cluster halves each CTA's rows (the per-term latency of the sweeps
// scales with them); it needs 16 SMs of one GPC free at once.  The device is
// asked once whether such a cluster of the backward sweep (the larger shared
// memory) for a 128^2 fp32 grid can be resident; otherwise 8 CTAs are used.
int advect_cluster_ctas() {
  static std::once_flag once;
  static int n = 8;
  std::call_once(once, [] {
    const void* k = (const void*)taylor_adjoint_kernel<float>;
    if (allow_max_smem(k) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    Geom g{};
    g.nx = g.ny = 128;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kMaxClusterCTAs, 1, 1);
    cfg.blockDim = dim3(kAdvThreads, 1, 1);
    cfg.dynamicSmemBytes = adv_layout<float>(g, true, kMaxClusterCTAs).total;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kMaxClusterCTAs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) == cudaSuccess && clusters >= 1) n = kMaxClusterCTAs;
    cudaGetLastError();
  });
  return n;
}

template <class K>
static cudaError_t cluster_launch(K kernel, size_t smem, cudaStream_t st, void** args) {
  cudaError_t e = allow_max_smem((const void*)kernel);
  if (e != cudaSuccess) return e;
  const int ncta = advect_cluster_ctas();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta, 1, 1);
  cfg.blockDim = dim3(kAdvThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}

template <class T>
cudaError_t launch_taylor_forward(const Geom& g, const T* vel, T* rho, int* K, double thresh, int kmax, int* err,
                                  cudaStream_t st) {
  if (kmax < 1 || kmax > kTaylorKmaxLimit) return cudaErrorInvalidValue;   // size of the dt/k table
  Geom gg = g;
  void* args[] = {&gg, (void*)&vel, (void*)&rho, (void*)&K, (void*)&thresh, (void*)&kmax, (void*)&err};
  return cluster_launch(taylor_forward_kernel<T>, adv_layout<T>(g, false, advect_cluster_ctas()).total, st, args);
}

template <class T>
cudaError_t launch_taylor_adjoint(const Geom& g, const T* vel, const T* rho, const int* K, const double* mterm,
                                  T* mu, const T* base, T alpha, T beta, T* out, T* powers, int kmax,
                                  int* err, cudaStream_t st, int s_end, T* mu_m1) {
  if (kmax < 1 || kmax > kTaylorKmaxLimit) return cudaErrorInvalidValue;   // size of the dt/k table
  if (s_end != 0 && s_end != 1) return cudaErrorInvalidValue;
  Geom gg = g;
  void* args[] = {&gg,          (void*)&vel,   (void*)&rho,  (void*)&K,   (void*)&mterm,  (void*)&mu,
                  (void*)&base, (void*)&alpha, (void*)&beta, (void*)&out, (void*)&powers, (void*)&kmax,
                  (void*)&s_end, (void*)&mu_m1, (void*)&err};
  return cluster_launch(taylor_adjoint_kernel<T>, adv_layout<T>(g, true, advect_cluster_ctas()).total, st, args);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the backward adjoint sweep.
//
// Some callers cannot allocate device memory when they need this sweep: a
// process that reserves its whole device-memory budget up front in its own
// pool (so a later cudaMalloc fails or is forbidden), or a latency-critical
// caller that cannot afford cudaMalloc's implicit device synchronisation.
// For them the sweep's only scratch -- the Taylor powers A^m rho_s, taylor_kmax
// cell fields -- lives in this file-scope device array instead of a buffer the
// problem allocates.  It is modest (4 MiB) and, being a module global, it is
// held on every GPU that loads the library until the process exits.  All
// calls share it, so calls that overlap on the GPU race; the powers need not
// start at zero (each is written before it is read).  A tail of 64 words after
// the powers holds the sweep's error word, cleared by each call before its
// launch.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocPowersFloats = (size_t)1 << 20;
constexpr size_t kNoAllocTailWords = 64;
static __device__ __align__(256) float g_noalloc_powers[kNoAllocPowersFloats + kNoAllocTailWords];

namespace {
std::mutex g_noalloc_mutex;
constexpr int kNoAllocMaxDevices = 256;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

// Device address of g_noalloc_powers on the current device, looked up once per
// device (the host-side symbol is only a stand-in, not a device address).
static cudaError_t noalloc_powers(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_powers);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace stc

extern "C" stc_status stc_adjoint_sweep_noalloc(int nx, int ny, int num_steps, double dt, int taylor_kmax,
                                                const float* vel, const float* rho, const int* K,
                                                const double* mterm, float* mu, const float* base, double alpha,
                                                double beta, float* out, void* cuda_stream) {
  using namespace stc;
  if (nx < 2 || ny < 2 || num_steps < 1 || !(dt > 0.0) || taylor_kmax < 1 || taylor_kmax > 256 || !vel || !rho ||
      !K || !mterm || !mu || !out) {
    set_last_error("stc_adjoint_sweep_noalloc: invalid argument");
    return STC_ERR_INVALID_ARG;
  }
  const size_t need = (size_t)taylor_kmax * (size_t)nx * (size_t)ny;
  if (need > kNoAllocPowersFloats) {
    set_last_error("stc_adjoint_sweep_noalloc: taylor_kmax * nx * ny exceeds the fixed scratch of 1048576 floats");
    return STC_ERR_INVALID_ARG;
  }
  Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.N = num_steps;
  g.Fx = ny * (nx + 1);
  g.F = g.Fx + (ny + 1) * nx;
  g.C = nx * ny;
  g.dim = 2;
  g.nz = 1;
  g.Fy = (ny + 1) * nx;
  g.Fxy = g.F;
  g.h = 1.0 / nx;
  g.ih = (double)nx;
  g.dt = dt;
  g.idt = 1.0 / dt;
  g.a = 0.0;
  g.lm = 0.0;
  g.omega = 1.0;
  g.self_adv = 1;
  set_fp32_copies(g);
  if (!advect_supported(g)) {
    set_last_error("stc_adjoint_sweep_noalloc: grid too large for the on-chip sweep");
    return STC_ERR_UNSUPPORTED;
  }
  float* scratch = nullptr;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = noalloc_powers(&scratch);
  int* err = scratch ? reinterpret_cast<int*>(scratch + kNoAllocPowersFloats) : nullptr;
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_taylor_adjoint<float>(g, vel, rho, K, mterm, mu, base, float(alpha), float(beta), out, scratch,
                                     taylor_kmax, err, st);
  // the error word comes back on the caller's stream (pageable host memory:
  // no allocation), so the call returns once the sweep has finished
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return STC_ERR_CUDA;
  }
  if (herr & DEV_TAYLOR_KMAX) {
    set_last_error("stc_adjoint_sweep_noalloc: a Taylor order in K lies outside 1..taylor_kmax");
    return STC_ERR_DIVERGED;
  }
  return STC_OK;
}

namespace stc {

#define STC_ADV_INST(T)                                                                                         \
  template cudaError_t launch_taylor_forward<T>(const Geom&, const T*, T*, int*, double, int, int*,           \
                                                cudaStream_t);                                                \
  template cudaError_t launch_taylor_adjoint<T>(const Geom&, const T*, const T*, const int*, const double*, T*, \
                                                const T*, T, T, T*, T*, int, int*, cudaStream_t, int, T*);     \
  template void launch_metric<T>(const Geom&, const T*, const double*, double, int, double, double*, double*,   \
                                 double*, cudaStream_t);
STC_ADV_INST(float)
STC_ADV_INST(double)

}  // namespace stc
