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

#include "../../include/stc.h"
#include "stc_internal.cuh"
#include "stc_kernels.h"

namespace cg = cooperative_groups;

namespace stc {

struct Slab {
  int r0, r1, rpc;  // owned rows [r0, r1), rows per CTA
};

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// QUICK face value (Leonard): upwind U, downwind D, far-upwind UU; v = 0 gives
// the mean of both one-sided values (subgradient convention).
template <class T>
__device__ __forceinline__ T quick(T vel, T tL, T tR, T tLL, T tRR) {
  const T pos = (T(6) * tL + T(3) * tR - tLL) * T(0.125);
  const T neg = (T(6) * tR + T(3) * tL - tRR) * T(0.125);
  if (vel > T(0)) return pos;
  if (vel < T(0)) return neg;
  return T(0.5) * (pos + neg);
}

// buffer with halo: row jj (clamped to the grid) of a slab buffer
template <class T>
__device__ __forceinline__ T buf_at(const Geom& g, const Slab& s, const T* b, int jj, int ii) {
  jj = clampi(jj, 0, g.ny - 1);
  ii = clampi(ii, 0, g.nx - 1);
  return b[(jj - s.r0 + 2) * g.nx + ii];
}

// (A(v) t)_c at own cell (j,i); vxs holds x-faces of rows [r0, r1),
// vys y-faces of rows [r0 - 1, r0 + rpc + 1] (offset 1).
template <class T>
__device__ T apply_A(const Geom& g, const Slab& s, const T* b, const T* vxs, const T* vys, int j, int i) {
  T fl = T(0), fr = T(0), fb = T(0), ft = T(0);
  const int lr = j - s.r0;
  if (i >= 1) {
    T v = vxs[lr * (g.nx + 1) + i];
    if (v != T(0))
      fl = v * quick(v, buf_at(g, s, b, j, i - 1), buf_at(g, s, b, j, i), buf_at(g, s, b, j, i - 2),
                     buf_at(g, s, b, j, i + 1));
  }
  if (i + 1 <= g.nx - 1) {
    T v = vxs[lr * (g.nx + 1) + i + 1];
    if (v != T(0))
      fr = v * quick(v, buf_at(g, s, b, j, i), buf_at(g, s, b, j, i + 1), buf_at(g, s, b, j, i - 1),
                     buf_at(g, s, b, j, i + 2));
  }
  if (j >= 1) {
    T v = vys[(j - s.r0 + 1) * g.nx + i];
    if (v != T(0))
      fb = v * quick(v, buf_at(g, s, b, j - 1, i), buf_at(g, s, b, j, i), buf_at(g, s, b, j - 2, i),
                     buf_at(g, s, b, j + 1, i));
  }
  if (j + 1 <= g.ny - 1) {
    T v = vys[(j + 1 - s.r0 + 1) * g.nx + i];
    if (v != T(0))
      ft = v * quick(v, buf_at(g, s, b, j, i), buf_at(g, s, b, j + 1, i), buf_at(g, s, b, j - 1, i),
                     buf_at(g, s, b, j + 2, i));
  }
  return -T(g.ih) * (fr - fl + ft - fb);
}

// weight of cell c in the QUICK stencil of the face between cells lo = f-1 and
// hi = f (along one axis of n cells) for velocity sign of v
template <class T>
__device__ __forceinline__ T quick_weight(T v, int f, int c, int n) {
  const int lo = f - 1, hi = f;
  T w = T(0);
  if (v > T(0)) {
    if (lo == c) w += T(0.75);
    if (hi == c) w += T(0.375);
    if (clampi(f - 2, 0, n - 1) == c) w -= T(0.125);
  } else if (v < T(0)) {
    if (hi == c) w += T(0.75);
    if (lo == c) w += T(0.375);
    if (clampi(f + 1, 0, n - 1) == c) w -= T(0.125);
  }
  return w;
}

// (A(v)^T w)_c at own cell (j,i): A^T = -R_up^T diag(v) D^T, so each face f
// whose upwind stencil contains c contributes weight * v_f * (w_hi - w_lo)/h.
template <class T>
__device__ T apply_AT(const Geom& g, const Slab& s, const T* b, const T* vxs, const T* vys, int j, int i) {
  T acc = T(0);
  const int lr = j - s.r0;
#pragma unroll
  for (int d = -1; d <= 2; ++d) {
    const int f = i + d;
    if (f >= 1 && f <= g.nx - 1) {
      T v = vxs[lr * (g.nx + 1) + f];
      T w = quick_weight(v, f, i, g.nx);
      if (w != T(0)) acc += w * v * (buf_at(g, s, b, j, f) - buf_at(g, s, b, j, f - 1));
    }
  }
#pragma unroll
  for (int d = -1; d <= 2; ++d) {
    const int f = j + d;
    if (f >= 1 && f <= g.ny - 1) {
      T v = vys[(f - s.r0 + 1) * g.nx + i];
      T w = quick_weight(v, f, j, g.ny);
      if (w != T(0)) acc += w * v * (buf_at(g, s, b, f, i) - buf_at(g, s, b, f - 1, i));
    }
  }
  return acc * T(g.ih);
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

template <class T>
__device__ void load_faces(const Geom& g, const Slab& s, const T* vel, T* vxs, T* vys) {
  const int nx = g.nx;
  const int nrx = s.r1 - s.r0;
  for (int e = threadIdx.x; e < nrx * (nx + 1); e += blockDim.x) vxs[e] = vel[(size_t)s.r0 * (nx + 1) + e];
  // y-face rows [r0 - 1, r1 + 1] clipped to [0, ny]
  const int nry = s.rpc + 3;
  for (int e = threadIdx.x; e < nry * nx; e += blockDim.x) {
    const int q = e / nx, i = e - q * nx;
    const int jj = s.r0 - 1 + q;
    vys[e] = (jj >= 0 && jj <= g.ny && s.r1 > s.r0) ? vel[g.Fx + (size_t)jj * nx + i] : T(0);
  }
}

template <class T>
struct AdvLayout {
  size_t buf, vx, vy, gx, gy;  // element counts of the T arrays
  size_t cm_off;               // byte offset of the fp64 cluster-max slots (16-byte aligned)
  size_t total;                // bytes
};

template <class T>
__host__ __device__ inline AdvLayout<T> adv_layout(const Geom& g, bool adjoint) {
  const int rpc = (g.ny + kClusterCTAs - 1) / kClusterCTAs;
  AdvLayout<T> L;
  L.buf = (size_t)(rpc + 4) * g.nx;
  L.vx = (size_t)rpc * (g.nx + 1);
  L.vy = (size_t)(rpc + 3) * g.nx;
  L.gx = adjoint ? (size_t)rpc * (g.nx + 1) : 0;
  L.gy = adjoint ? (size_t)(rpc + 1) * g.nx : 0;
  L.cm_off = ((2 * L.buf + L.vx + L.vy + L.gx + L.gy) * sizeof(T) + 15) / 16 * 16;
  L.total = L.cm_off + 2 * kClusterCTAs * sizeof(double);
  return L;
}

__device__ __forceinline__ Slab make_slab(const Geom& g, int rank) {
  Slab s;
  s.rpc = (g.ny + kClusterCTAs - 1) / kClusterCTAs;
  s.r0 = rank * s.rpc;
  if (s.r0 > g.ny) s.r0 = g.ny;
  s.r1 = s.r0 + s.rpc;
  if (s.r1 > g.ny) s.r1 = g.ny;
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  return m;
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
  const Slab s = make_slab(g, rank);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const AdvLayout<T> L = adv_layout<T>(g, false);
  T* tb0 = reinterpret_cast<T*>(smem_raw);
  T* tb1 = tb0 + L.buf;
  T* vxs = tb1 + L.buf;
  T* vys = vxs + L.vx;
  double* cmax = reinterpret_cast<double*>(smem_raw + L.cm_off);
  __shared__ double red[32];
  const int nown = (s.r1 - s.r0) * g.nx;

  T acc[kAdvMaxCellsPerThread], cmp[kAdvMaxCellsPerThread];
#pragma unroll
  for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    acc[q] = (e < nown) ? rho[(size_t)s.r0 * g.nx + e] : T(0);
    cmp[q] = T(0);
  }
  int kfail = 0;
  for (int st = 0; st < g.N; ++st) {
    // t_0 = rho_st into tb0 own rows, its halo pushed; faces of v_st
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) tb0[2 * g.nx + e] = acc[q];
    }
    load_faces(g, s, vel + (size_t)st * g.F, vxs, vys);
    __syncthreads();
    halo_push(cl, g, s, tb0, rank);
    cl.sync();
    T* cur = tb0;
    T* nxt = tb1;
    int K = kmax;
    bool done = false;
    for (int k = 1; k <= kmax; ++k) {
      const T ck = T(g.dt / k);
      double lmax = 0.0;
#pragma unroll
      for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < nown) {
          const int j = s.r0 + e / g.nx, i = e % g.nx;
          const T t = ck * apply_A(g, s, cur, vxs, vys, j, i);
          nxt[2 * g.nx + e] = t;
          // two-sum accumulation of the series
          const T sum = acc[q] + t;
          const T bb = sum - acc[q];
          cmp[q] += (acc[q] - (sum - bb)) + (t - bb);
          acc[q] = sum;
          lmax = fmax(lmax, fabs((double)t));
        }
      }
      const double bm = block_max(lmax, red);   // also orders the nxt writes before the push
      halo_push(cl, g, s, nxt, rank);
      if (threadIdx.x < kClusterCTAs)
        *cl.map_shared_rank(cmax + (k & 1) * kClusterCTAs + rank, (int)threadIdx.x) = bm;
      cl.sync();
      double gm = 0.0;
#pragma unroll
      for (int r = 0; r < kClusterCTAs; ++r) gm = fmax(gm, cmax[(k & 1) * kClusterCTAs + r]);
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
      if (gm < thresh) {
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
// backward sweep.  For s = N-1 .. 1 with mu_s known:
//   powers P_m = A^m rho_s (m < K_s) -> global scratch
//   Horner  w_{K-1} = c_K mu, w_{m-1} = c_m mu + A^T w_m  (c_m = dt^m / m!)
//   grad    = sum_m B(P_m)^T w_m  = (dA[rho_s, v_s]/dv_s)^T mu_s
//   T^T mu  = w_{-1};  mu_{s-1} = T^T mu_s - m_s
// B(x)^T w at a face = QUICK(x)_face * (w_hi - w_lo) / h.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kAdvThreads, 1)
taylor_adjoint_kernel(Geom g, const T* __restrict__ vel, const T* __restrict__ rho, const int* __restrict__ Ks,
                      const double* __restrict__ mterm, T* mu, const T* __restrict__ base, T alpha, T beta,
                      T* out, T* powers, int kmax) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const Slab s = make_slab(g, rank);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const AdvLayout<T> L = adv_layout<T>(g, true);
  T* tb0 = reinterpret_cast<T*>(smem_raw);
  T* tb1 = tb0 + L.buf;
  T* vxs = tb1 + L.buf;
  T* vys = vxs + L.vx;
  T* gxs = vys + L.vy;
  T* gys = gxs + L.gx;
  const int nx = g.nx;
  const int nown = (s.r1 - s.r0) * nx;
  const int ngx = (s.r1 - s.r0) * (nx + 1);
  const int ngy = (s.r1 - s.r0) * nx;

  T m[kAdvMaxCellsPerThread];
#pragma unroll
  for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    m[q] = (e < nown) ? T(-mterm[(size_t)g.N * g.C + (size_t)s.r0 * nx + e]) : T(0);
  }
  for (int st = g.N - 1; st >= 1; --st) {
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
    if (K < 1) K = 1;
    if (K > kmax) K = kmax;
    const T* vs = vel + (size_t)st * g.F;
    const T* rs = rho + (size_t)st * g.C;
    load_faces(g, s, vs, vxs, vys);
    // powers P_1 .. P_{K-1}
    for (int e = threadIdx.x; e < nown; e += blockDim.x) tb0[2 * nx + e] = rs[(size_t)s.r0 * nx + e];
    __syncthreads();
    halo_push(cl, g, s, tb0, rank);
    T* cur = tb0;
    T* nxt = tb1;
    for (int k = 1; k < K; ++k) {
      cl.sync();
      for (int e = threadIdx.x; e < nown; e += blockDim.x) {
        const int j = s.r0 + e / nx, i = e % nx;
        const T t = apply_A(g, s, cur, vxs, vys, j, i);
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
    // c_K = dt^K / K!
    double cK = 1.0;
    for (int k = 1; k <= K; ++k) cK *= g.dt / k;
    cl.sync();  // powers visible to the cluster; everyone done with tb buffers
    cur = tb0;
    nxt = tb1;
#pragma unroll
    for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < nown) cur[2 * nx + e] = T(cK) * m[q];
    }
    __syncthreads();
    halo_push(cl, g, s, cur, rank);
    double cm = cK;
    for (int mm = K - 1; mm >= 0; --mm) {
      cl.sync();
      const T* P = (mm == 0) ? rs : powers + (size_t)mm * g.C;
      // grad += B(P_m)^T w_m on own faces
      for (int e = threadIdx.x; e < ngx; e += blockDim.x) {
        const int j = s.r0 + e / (nx + 1), i = e % (nx + 1);
        if (i >= 1 && i <= nx - 1) {
          const T v = vxs[e];
          const T* Pr = P + (size_t)j * nx;
          const T xf = quick(v, Pr[i - 1], Pr[i], Pr[clampi(i - 2, 0, nx - 1)], Pr[clampi(i + 1, 0, nx - 1)]);
          gxs[e] += xf * (buf_at(g, s, cur, j, i) - buf_at(g, s, cur, j, i - 1)) * T(g.ih);
        }
      }
      for (int e = threadIdx.x; e < ngy; e += blockDim.x) {
        const int j = s.r0 + e / nx, i = e % nx;
        if (j >= 1 && j <= g.ny - 1) {
          const T v = vys[(j - s.r0 + 1) * nx + i];
          const T xf = quick(v, P[(size_t)(j - 1) * nx + i], P[(size_t)j * nx + i],
                             P[(size_t)clampi(j - 2, 0, g.ny - 1) * nx + i],
                             P[(size_t)clampi(j + 1, 0, g.ny - 1) * nx + i]);
          gys[e] += xf * (buf_at(g, s, cur, j, i) - buf_at(g, s, cur, j - 1, i)) * T(g.ih);
        }
      }
      // w_{m-1} = c_m mu + A^T w_m with c_m = c_{m+1} (m+1) / dt  (c_0 = 1: T^T mu)
      const double cprev = (mm == 0) ? 1.0 : cm * (mm + 1) / g.dt;
#pragma unroll
      for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < nown) {
          const int j = s.r0 + e / nx, i = e % nx;
          nxt[2 * nx + e] = T(cprev) * m[q] + apply_AT(g, s, cur, vxs, vys, j, i);
        }
      }
      cm = cprev;
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
#pragma unroll
  for (int q = 0; q < kAdvMaxCellsPerThread; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    if (e < nown) mu[(size_t)s.r0 * nx + e] = m[q];
  }
  cl.sync();
}

// ---------------------------------------------------------------------------
// keyframe metric: m = c * sum_l G_l^T G_l (rho - rho*), separable Gaussian
// filters (sigma_l = sigma0 2^l cells, taps to ceil(3 sigma), normalised,
// clamp-to-edge).  G^T is evaluated as a gather of the clamped-tap matrix.
// ---------------------------------------------------------------------------
__global__ void blur_kernel(int nx, int ny, int axis, int transpose, double sigma, const double* __restrict__ in,
                            double* out, double scale, int accumulate) {
  extern __shared__ double w[];
  const int R = (int)ceil(3.0 * sigma);
  const int nt = 2 * R + 1;
  __shared__ double wsum;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double d = t - R;
    w[t] = exp(-d * d / (2.0 * sigma * sigma));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += w[t];
    wsum = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nt; t += blockDim.x) w[t] /= wsum;
  __syncthreads();
  const int n = axis == 0 ? nx : ny;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nx * ny; e += gridDim.x * blockDim.x) {
    const int j = e / nx, i = e % nx;
    const int a = axis == 0 ? i : j;
    auto at = [&](int b) { return axis == 0 ? in[j * nx + b] : in[b * nx + i]; };
    double acc = 0.0;
    if (!transpose) {
      for (int t = -R; t <= R; ++t) acc += w[t + R] * at(clampi(a + t, 0, n - 1));
    } else {
      // (G^T y)_a = sum_b G[b,a] y_b, G[b,a] = sum_t w_t [clamp(b+t) == a]
      const int lo = a - R < 0 ? 0 : a - R, hi = a + R > n - 1 ? n - 1 : a + R;
      for (int b = lo; b <= hi; ++b) {
        double gba = 0.0;
        if (a == 0 && a == n - 1) {
          gba = 1.0;
        } else if (a == 0) {
          for (int t = -R; t <= -b; ++t) gba += w[t + R];
        } else if (a == n - 1) {
          for (int t = n - 1 - b; t <= R; ++t) gba += w[t + R];
        } else {
          gba = w[a - b + R];
        }
        acc += gba * at(b);
      }
    }
    acc *= scale;
    if (accumulate) out[e] += acc;
    else out[e] = acc;
  }
}

template <class T>
__global__ void metric_diff_kernel(const T* __restrict__ rho, const double* __restrict__ star, double* d, int C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C; e += gridDim.x * blockDim.x)
    d[e] = (double)rho[e] - star[e];
}

__global__ void scale_kernel(const double* __restrict__ in, double* out, double c, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) out[e] = c * in[e];
}

// tmp0: C doubles, tmp1: 2C doubles
template <class T>
void launch_metric(const Geom& g, const T* rho_s, const double* star, double c, int levels, double sigma0,
                   double* out, double* tmp0, double* tmp1, cudaStream_t st) {
  const int C = g.C;
  const int tpb = 256;
  const unsigned nb = (unsigned)((C + tpb - 1) / tpb);
  metric_diff_kernel<T><<<nb, tpb, 0, st>>>(rho_s, star, tmp0, C);
  if (levels <= 0) {
    scale_kernel<<<nb, tpb, 0, st>>>(tmp0, out, c, C);   // C_i = c_i I
    return;
  }
  cudaMemsetAsync(out, 0, sizeof(double) * C, st);
  for (int l = 0; l < levels; ++l) {
    const double sig = sigma0 * (double)(1 << l);
    const int R = (int)ceil(3.0 * sig);
    const size_t sm = sizeof(double) * (2 * R + 1);
    blur_kernel<<<nb, tpb, sm, st>>>(g.nx, g.ny, 0, 0, sig, tmp0, tmp1, 1.0, 0);        // G_x
    blur_kernel<<<nb, tpb, sm, st>>>(g.nx, g.ny, 1, 0, sig, tmp1, tmp1 + C, 1.0, 0);    // G_y
    blur_kernel<<<nb, tpb, sm, st>>>(g.nx, g.ny, 1, 1, sig, tmp1 + C, tmp1, 1.0, 0);    // G_y^T
    blur_kernel<<<nb, tpb, sm, st>>>(g.nx, g.ny, 0, 1, sig, tmp1, out, c, 1);           // += c G_x^T
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
bool advect_supported(const Geom& g) {
  const int rpc = (g.ny + kClusterCTAs - 1) / kClusterCTAs;
  return g.nx >= 2 && g.ny >= 2 && rpc * g.nx <= kAdvThreads * kAdvMaxCellsPerThread;
}
size_t advect_smem_forward(const Geom& g, size_t tsize) {
  return tsize == 4 ? adv_layout<float>(g, false).total : adv_layout<double>(g, false).total;
}
size_t advect_smem_adjoint(const Geom& g, size_t tsize) {
  return tsize == 4 ? adv_layout<float>(g, true).total : adv_layout<double>(g, true).total;
}

template <class K>
static cudaError_t cluster_launch(K kernel, size_t smem, cudaStream_t st, void** args) {
  cudaError_t e = cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCTAs, 1, 1);
  cfg.blockDim = dim3(kAdvThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCTAs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}

template <class T>
cudaError_t launch_taylor_forward(const Geom& g, const T* vel, T* rho, int* K, double thresh, int kmax, int* err,
                                  cudaStream_t st) {
  Geom gg = g;
  void* args[] = {&gg, (void*)&vel, (void*)&rho, (void*)&K, (void*)&thresh, (void*)&kmax, (void*)&err};
  return cluster_launch(taylor_forward_kernel<T>, adv_layout<T>(g, false).total, st, args);
}

template <class T>
cudaError_t launch_taylor_adjoint(const Geom& g, const T* vel, const T* rho, const int* K, const double* mterm,
                                  T* mu, const T* base, T alpha, T beta, T* out, T* powers, int kmax,
                                  cudaStream_t st) {
  Geom gg = g;
  void* args[] = {&gg,          (void*)&vel,  (void*)&rho,   (void*)&K,   (void*)&mterm,  (void*)&mu,
                  (void*)&base, (void*)&alpha, (void*)&beta, (void*)&out, (void*)&powers, (void*)&kmax};
  return cluster_launch(taylor_adjoint_kernel<T>, adv_layout<T>(g, true).total, st, args);
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
// calls share it, so calls that overlap on the GPU race; nothing in it needs
// to start at zero (each power is written before it is read).
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocPowersFloats = (size_t)1 << 20;
static __device__ __align__(256) float g_noalloc_powers[kNoAllocPowersFloats];

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
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.N = num_steps;
  g.Fx = ny * (nx + 1);
  g.F = g.Fx + (ny + 1) * nx;
  g.C = nx * ny;
  g.h = 1.0 / nx;
  g.ih = (double)nx;
  g.dt = dt;
  g.idt = 1.0 / dt;
  g.a = 0.0;
  g.lm = 0.0;
  g.omega = 1.0;
  g.self_adv = 1;
  if (!advect_supported(g)) {
    set_last_error("stc_adjoint_sweep_noalloc: grid too large for the on-chip sweep");
    return STC_ERR_UNSUPPORTED;
  }
  float* scratch = nullptr;
  cudaError_t e = noalloc_powers(&scratch);
  if (e == cudaSuccess)
    e = launch_taylor_adjoint<float>(g, vel, rho, K, mterm, mu, base, float(alpha), float(beta), out, scratch,
                                     taylor_kmax, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return STC_ERR_CUDA;
  }
  return STC_OK;
}

namespace stc {

#define STC_ADV_INST(T)                                                                                         \
  template cudaError_t launch_taylor_forward<T>(const Geom&, const T*, T*, int*, double, int, int*,           \
                                                cudaStream_t);                                                \
  template cudaError_t launch_taylor_adjoint<T>(const Geom&, const T*, const T*, const int*, const double*, T*, \
                                                const T*, T, T, T*, T*, int, cudaStream_t);                    \
  template void launch_metric<T>(const Geom&, const T*, const double*, double, int, double, double*, double*,   \
                                 double*, cudaStream_t);
STC_ADV_INST(float)
STC_ADV_INST(double)

}  // namespace stc
