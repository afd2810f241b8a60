// Passive advection by the truncated Taylor exponential (Sec. 3.1, Eq. Adv),
// the backward adjoint sweep (Eq. KKTPO, Alg. 1) and the keyframe metric
// (Sec. 4.1) on the 3D grid.
//
// A 3D step has too many cells for one cluster's shared memory, so each sweep
// is ONE cooperative launch over the whole GPU (all CTAs resident): the
// threads stride over the cells, the series terms live in two L2-resident
// global buffers, and a grid-wide barrier separates consecutive terms.  The
// barrier is this file's own (an arrival counter and a generation word) with
// an iteration limit: a CTA that waits too long sets DEV_BARRIER_TIMEOUT and
// returns, so a fault never becomes a hang.  Buffers that other CTAs write
// during the launch are read with ld.global.cg (L2, never a stale L1 line).
#include <mutex>

#include "grid3d.cuh"
#include "stc_kernels.h"

namespace stc {
namespace {

using namespace g3;

constexpr int kAdv3Threads = 512;
constexpr long long kBarrierSpinLimit = 1LL << 24;   // >= ~1 s with the back-off below

// grid barrier: bar[0] arrivals, bar[1] generation.  Returns false on timeout.
__device__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > kBarrierSpinLimit) {
          ok = 0;
          atomicOr(err, DEV_BARRIER_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <class T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

__device__ __forceinline__ void atomic_max_nonneg3(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// QUICK coefficients of (lo, hi, lo-1, hi+1), as in the 2D sweeps
template <class T>
__device__ __forceinline__ void quick_coef3(T v, T c[4]) {
  const bool pos = v > T(0), neg = v < T(0);
  c[0] = pos ? T(0.75) : (neg ? T(0.375) : T(0.5625));
  c[1] = pos ? T(0.375) : (neg ? T(0.75) : T(0.5625));
  c[2] = pos ? T(-0.125) : (neg ? T(0) : T(-0.0625));
  c[3] = pos ? T(0) : (neg ? T(-0.125) : T(-0.0625));
}

struct Axis {
  int n, stride;   // cells along the axis, cell-index stride
};
__device__ __forceinline__ Axis axis_of(const Geom& g, int a) {
  return a == 0 ? Axis{g.nx, 1} : (a == 1 ? Axis{g.ny, g.nx} : Axis{g.nz, g.nx * g.ny});
}
// face of axis a at position p (0..n) along it, through the cell `c0` whose
// coordinate along a is 0 (the other two coordinates fixed)
__device__ __forceinline__ int face_at(const Geom& g, int a, int k, int j, int i) {
  return a == 0 ? xf(g, k, j, i) : (a == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
}

// position p +- d of an axis line: clamped to the wall cells, or wrapped
__device__ __forceinline__ int line_pos(const Geom& g, int p, int n) {
  if (g.periodic) return p < 0 ? p + n : (p >= n ? p - n : p);
  return p < 0 ? 0 : (p > n - 1 ? n - 1 : p);
}

// QUICK face value of cell field t at the face p along axis a of the line
// through cell c0 (the line's first cell), normal velocity vf: lower cell p-1,
// upper cell p, far cells p-2 and p+1 (clamped at walls, wrapped if periodic)
template <class T>
__device__ __forceinline__ T quick_face(const Geom& g, const T* t, int c0, Axis ax, int p, T vf) {
  T c[4];
  quick_coef3(vf, c);
  const int lo = line_pos(g, p - 1, ax.n), hi = line_pos(g, p, ax.n);
  const int llo = line_pos(g, p - 2, ax.n), hhi = line_pos(g, p + 1, ax.n);
  return c[0] * ldcg(t + c0 + lo * ax.stride) + c[1] * ldcg(t + c0 + hi * ax.stride) +
         c[2] * ldcg(t + c0 + llo * ax.stride) + c[3] * ldcg(t + c0 + hhi * ax.stride);
}

// (A(v) t)_c = -(1/h) sum_a (F_{c+1/2} - F_{c-1/2}), F_f = v_f QUICK(t)_f, 0 on walls
template <class T>
__device__ T apply_A(const Geom& g, const T* v, const T* t, int k, int j, int i) {
  const int crd[3] = {i, j, k};
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Axis ax = axis_of(g, a);
    const int p = crd[a];
    const int c0 = cid(g, k, j, i) - p * ax.stride;
    const int fm = a == 0 ? face_at(g, 0, k, j, i) : (a == 1 ? face_at(g, 1, k, j, i) : face_at(g, 2, k, j, i));
    const int fp = a == 0 ? face_at(g, 0, k, j, i + 1) : (a == 1 ? face_at(g, 1, k, j + 1, i) : face_at(g, 2, k + 1, j, i));
    T Fp = T(0), Fm = T(0);
    if (g.periodic || p + 1 <= ax.n - 1) {
      const T vf = ld(v + fp);
      Fp = vf * quick_face(g, t, c0, ax, p + 1, vf);
    }
    if (g.periodic || p >= 1) {
      const T vf = ld(v + fm);
      Fm = vf * quick_face(g, t, c0, ax, p, vf);
    }
    acc += Fp - Fm;
  }
  return -pick<T>(g.ih, g.ihf) * acc;
}

// (A(v)^T w)_c: sum over the faces f of each axis line whose QUICK stencil
// holds c of coef(f, c) E_f, E_f = v_f (w_hi - w_lo) / h (clamped stencils
// included: face 1 also reaches cell 0 through lo-1, face n-1 cell n-1 through
// hi+1; on a periodic axis the faces p-1 .. p+2 wrap)
template <class T>
__device__ T apply_AT(const Geom& g, const T* v, const T* w, int k, int j, int i) {
  const int crd[3] = {i, j, k};
  const T ih = pick<T>(g.ih, g.ihf);
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Axis ax = axis_of(g, a);
    const int p = crd[a];
    const int c0 = cid(g, k, j, i) - p * ax.stride;
#pragma unroll
    for (int d = -1; d <= 2; ++d) {
      int f = p + d;     // face position along the axis
      if (g.periodic) f = f < 0 ? f + ax.n : (f >= ax.n ? f - ax.n : f);
      else if (f < 1 || f > ax.n - 1) continue;
      const int fk = a == 2 ? f : k, fj = a == 1 ? f : j, fi = a == 0 ? f : i;
      const T vf = ld(v + face_at(g, a, fk, fj, fi));
      T c[4];
      quick_coef3(vf, c);
      const int lo = line_pos(g, f - 1, ax.n), hi = f;
      const int llo = line_pos(g, f - 2, ax.n), hhi = line_pos(g, f + 1, ax.n);
      const T E = vf * (ldcg(w + c0 + hi * ax.stride) - ldcg(w + c0 + lo * ax.stride)) * ih;
      T cf = T(0);
      if (lo == p) cf += c[0];
      if (hi == p) cf += c[1];
      if (llo == p) cf += c[2];
      if (hhi == p) cf += c[3];
      acc += cf * E;
    }
  }
  return acc;
}

__device__ __forceinline__ void cell_coords(const Geom& g, int e, int& k, int& j, int& i) {
  i = e % g.nx;
  const int r = e / g.nx;
  j = r % g.ny;
  k = r / g.ny;
}

template <class T>
__device__ __forceinline__ T block_max3(T v) {
  __shared__ T red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T m = T(0);
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  __syncthreads();
  return m;   // valid in thread 0
}

// scratch layout: tb0 [C], tb1 [C], cmp [C] (T), then the barrier words and
// three fp64 max slots at a 16-byte-aligned offset
struct Adv3Scratch {
  size_t tb0, tb1, cmp, ctl;   // element offsets (T) / byte offset of the control block
};
template <class T>
__host__ __device__ inline size_t adv3_ctl_offset(int C) {
  return ((3 * (size_t)C * sizeof(T)) + 255) & ~(size_t)255;
}

// forward sweep: rho_{s+1} = sum_{k<=K} (dt^k/k!) A(v_s)^k rho_s, K the first
// order with max|t_k| < thresh (the small term included); compensated sum
template <class T>
__global__ void __launch_bounds__(kAdv3Threads)
taylor_forward3_kernel(Geom g, const T* __restrict__ vel, T* rho, int* Ks, double thresh, int kmax, int* err,
                       unsigned char* scratch) {
  __shared__ T dtk[kTaylorKmaxLimit + 1];
  __shared__ double gm_s;
  for (int k = threadIdx.x; k <= kmax; k += blockDim.x) dtk[k] = k == 0 ? T(1) : T(g.dt / (double)k);
  const int C = g.C;
  T* tb0 = reinterpret_cast<T*>(scratch);
  T* tb1 = tb0 + C;
  T* cmp = tb1 + C;
  unsigned* bar = reinterpret_cast<unsigned*>(scratch + adv3_ctl_offset<T>(C));
  double* slots = reinterpret_cast<double*>(bar + 4);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  __syncthreads();
  int tau = 0, kfail = 0;
  for (int st = 0; st < g.N; ++st) {
    const T* vs = vel + (size_t)st * g.F;
    T* acc = rho + (size_t)(st + 1) * C;
    const T* r0 = rho + (size_t)st * C;
    for (int e = tid; e < C; e += nth) {
      const T x = ldcg(r0 + e);
      tb0[e] = x;
      acc[e] = x;
      cmp[e] = T(0);
    }
    if (!grid_barrier(bar, err)) return;
    T* cur = tb0;
    T* nxt = tb1;
    int K = kmax;
    bool done = false;
    for (int k = 1; k <= kmax; ++k) {
      T lmax = T(0);
      for (int e = tid; e < C; e += nth) {
        int ck, cj, ci;
        cell_coords(g, e, ck, cj, ci);
        const T t = dtk[k] * apply_A(g, vs, cur, ck, cj, ci);
        nxt[e] = t;
        const T a = acc[e];
        const T sum = a + t;
        const T bb = sum - a;
        cmp[e] += (a - (sum - bb)) + (t - bb);
        acc[e] = sum;
        lmax = fmax(lmax, fabs(t));
      }
      const T bm = block_max3(lmax);
      if (threadIdx.x == 0) {
        atomic_max_nonneg3(slots + tau % 3, (double)bm);
        if (blockIdx.x == 0) slots[(tau + 1) % 3] = 0.0;
      }
      if (!grid_barrier(bar, err)) return;
      if (threadIdx.x == 0) gm_s = __ldcg(slots + tau % 3);
      __syncthreads();
      const double gm = gm_s;
      ++tau;
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
    for (int e = tid; e < C; e += nth) acc[e] += cmp[e];
    if (tid == 0) Ks[st] = K;
    // the next step reads rho_{st+1} of every cell
    if (!grid_barrier(bar, err)) return;
  }
  if (kfail && tid == 0) atomicOr(err, DEV_TAYLOR_KMAX);
}

// backward sweep, as the 2D kernel (scaled Horner over the series terms):
//   w'_{K-1} = (dt/K) mu,  w'_{m-1} = (dt/m)(mu + A^T w'_m),
//   grad = sum_m B(t_m)^T w'_m,  T^T mu = mu + A^T w'_0,
// with t_m = (dt^m/m!) A^m rho_s and B(x)^T w at a face = QUICK(x)_f (w_hi - w_lo)/h.
// out_s = alpha base_s + beta grad_s (s = 1..N-1); mu_{s-1} = T^T mu_s - m_s.
template <class T>
__global__ void __launch_bounds__(kAdv3Threads)
taylor_adjoint3_kernel(Geom g, const T* __restrict__ vel, const T* __restrict__ rho, const int* __restrict__ Ks,
                       const double* __restrict__ mterm, T* mu, const T* __restrict__ base, T alpha, T beta, T* out,
                       T* powers, int kmax, int* err, unsigned char* scratch, int s_end, T* mu_m1) {
  __shared__ T dtk[kTaylorKmaxLimit + 1];
  for (int k = threadIdx.x; k <= kmax; k += blockDim.x) dtk[k] = k == 0 ? T(1) : T(g.dt / (double)k);
  const int C = g.C, F = g.F;
  T* tb0 = reinterpret_cast<T*>(scratch);
  T* tb1 = tb0 + C;
  unsigned* bar = reinterpret_cast<unsigned*>(scratch + adv3_ctl_offset<T>(C));
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const T ih = pick<T>(g.ih, g.ihf);
  __syncthreads();
  // m = mu_{N-1} = -m_N, kept in mu's slab of the current step
  T* m = mu + (size_t)(g.N - 1) * C;
  for (int e = tid; e < C; e += nth) m[e] = T(-mterm[(size_t)g.N * C + e]);
  for (int st = g.N - 1; st >= s_end; --st) {
    m = mu + (size_t)st * C;
    int K = Ks[st];
    K = K < 1 ? 1 : (K > kmax ? kmax : K);
    const T* rs = rho + (size_t)st * C;
    const T* vs = vel + (size_t)st * F;
    // powers t_1 .. t_{K-1}
    for (int k = 1; k < K; ++k) {
      const T* src = k == 1 ? rs : powers + (size_t)(k - 1) * C;
      T* dst = powers + (size_t)k * C;
      for (int e = tid; e < C; e += nth) {
        int ck, cj, ci;
        cell_coords(g, e, ck, cj, ci);
        dst[e] = dtk[k] * apply_A(g, vs, src, ck, cj, ci);
      }
      if (!grid_barrier(bar, err)) return;
    }
    T* os = out + (size_t)st * F;
    const T* bs = base ? base + (size_t)st * F : nullptr;
    for (int f = tid; f < F; f += nth) os[f] = bs ? alpha * bs[f] : T(0);
    T* cur = tb0;
    T* nxt = tb1;
    for (int e = tid; e < C; e += nth) cur[e] = dtk[K] * m[e];
    if (!grid_barrier(bar, err)) return;
    for (int mm = K - 1; mm >= 0; --mm) {
      const T* P = mm == 0 ? rs : powers + (size_t)mm * C;
      // grad += beta B(t_mm)^T w'_mm on the interior faces
      for (int f = tid; f < F; f += nth) {
        int fk, fj, fi;
        const int a = face_coords(g, f, fk, fj, fi);
        if (!is_face(g, a, fk, fj, fi)) continue;
        const Axis ax = axis_of(g, a);
        const int p = a == 0 ? fi : (a == 1 ? fj : fk);
        const int c0 = cid(g, a == 2 ? 0 : fk, a == 1 ? 0 : fj, a == 0 ? 0 : fi);
        const T vf = ld(vs + f);
        const T q = quick_face(g, P, c0, ax, p, vf);
        const T d = (ldcg(cur + c0 + p * ax.stride) - ldcg(cur + c0 + line_pos(g, p - 1, ax.n) * ax.stride)) * ih;
        os[f] += beta * q * d;
      }
      const T fac = mm == 0 ? T(1) : dtk[mm];
      for (int e = tid; e < C; e += nth) {
        int ck, cj, ci;
        cell_coords(g, e, ck, cj, ci);
        nxt[e] = fac * (m[e] + apply_AT(g, vs, cur, ck, cj, ci));
      }
      if (!grid_barrier(bar, err)) return;
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    // mu_{st-1} = T^T mu_st - m_st (for st = 0: the adjoint density of step 0, into mu_m1)
    T* mprev = st > 0 ? mu + (size_t)(st - 1) * C : mu_m1;
    if (mprev)
      for (int e = tid; e < C; e += nth) mprev[e] = cur[e] - T(mterm[(size_t)st * C + e]);
    if (!grid_barrier(bar, err)) return;
  }
}

// ---------------------------------------------------------------------------
// keyframe metric m = c sum_l G_l^T G_l (rho - rho*), separable along three
// axes (weights and the clamped-tap transpose as the 2D blur kernel)
// ---------------------------------------------------------------------------
template <class Tc, class To>
__global__ void blur3_kernel(int nx, int ny, int nz, int axis, int transpose, double sigma, const Tc* __restrict__ in,
                             To* out, double scale, int accumulate, int periodic) {
  extern __shared__ double wsm3[];
  const int R = (int)ceil(3.0 * sigma);
  const int nt = 2 * R + 1;
  double* wd = wsm3;
  Tc* w = reinterpret_cast<Tc*>(wsm3 + nt);
  Tc* cw = w + nt;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) {
      const double d = t - R;
      s += exp(-d * d / (2.0 * sigma * sigma));
      wd[t] = s;                       // prefix sums of the raw weights
    }
  }
  __syncthreads();
  const double inv = 1.0 / wd[nt - 1];
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    w[t] = Tc((t > 0 ? wd[t] - wd[t - 1] : wd[0]) * inv);
    cw[t] = Tc(wd[t] * inv);
  }
  __syncthreads();
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const int stride = axis == 0 ? 1 : (axis == 1 ? nx : nx * ny);
  const int total = nx * ny * nz;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int crd = axis == 0 ? e % nx : (axis == 1 ? (e / nx) % ny : e / (nx * ny));
    const int base = e - crd * stride;
    auto at = [&](int b) { return in[base + b * stride]; };
    const int a = crd;
    Tc acc = Tc(0);
    if (periodic) {
      // circulant: G^T is the same filter with the taps reversed
      for (int t = -R; t <= R; ++t) {
        int b = (a + (transpose ? -t : t)) % n;
        b = b < 0 ? b + n : b;
        acc += w[t + R] * at(b);
      }
    } else if (!transpose) {
      for (int t = -R; t <= R; ++t) {
        int b = a + t;
        b = b < 0 ? 0 : (b > n - 1 ? n - 1 : b);
        acc += w[t + R] * at(b);
      }
    } else {
      const int lo = a - R < 0 ? 0 : a - R, hi = a + R > n - 1 ? n - 1 : a + R;
      if (n == 1) {
        acc = at(0);
      } else if (a == 0) {
        for (int b = lo; b <= hi; ++b) acc += cw[R - b] * at(b);
      } else if (a == n - 1) {
        for (int b = lo; b <= hi; ++b) {
          const int k0 = n - 2 - b + R;
          acc += (cw[2 * R] - (k0 >= 0 ? cw[k0] : Tc(0))) * at(b);
        }
      } else {
        for (int b = lo; b <= hi; ++b) acc += w[a - b + R] * at(b);
      }
    }
    const Tc val = acc * Tc(scale);
    if (accumulate) out[e] += To(val);
    else out[e] = To(val);
  }
}

template <class T>
__global__ void metric3_diff_kernel(const T* __restrict__ rho, const double* __restrict__ star, T* d, int C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C; e += gridDim.x * blockDim.x)
    d[e] = T((double)rho[e] - star[e]);
}

template <class T>
__global__ void metric3_scale_kernel(const T* __restrict__ in, double* out, double c, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) out[e] = c * (double)in[e];
}

struct CoopShape {
  int blocks;
  cudaError_t err;
};

// one cooperative grid: every SM, as many CTAs per SM as can be resident (<= 2)
template <class K>
CoopShape coop_shape(K kernel) {
  CoopShape s{0, cudaSuccess};
  int dev = 0, sms = 0, per = 0;
  s.err = cudaGetDevice(&dev);
  if (s.err == cudaSuccess) s.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (s.err == cudaSuccess)
    s.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)kernel, kAdv3Threads, 0);
  if (s.err != cudaSuccess) return s;
  if (per > 2) per = 2;
  if (per < 1) {
    s.err = cudaErrorLaunchOutOfResources;
    return s;
  }
  s.blocks = sms * per;
  return s;
}

template <class K>
cudaError_t coop_launch(K kernel, int blocks, cudaStream_t st, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(kAdv3Threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}

}  // namespace

size_t advect3_scratch_bytes(const Geom& g, size_t tsize) {
  const size_t ctl = tsize == 4 ? adv3_ctl_offset<float>(g.C) : adv3_ctl_offset<double>(g.C);
  return ctl + 4 * sizeof(unsigned) + 3 * sizeof(double) + 64;
}

template <class T>
cudaError_t launch_taylor_forward3(const Geom& g, const T* vel, T* rho, int* K, double thresh, int kmax, int* err,
                                   void* scratch, cudaStream_t st) {
  if (kmax < 1 || kmax > kTaylorKmaxLimit || !scratch) return cudaErrorInvalidValue;
  static std::once_flag once;
  static CoopShape shape;
  std::call_once(once, [] { shape = coop_shape(taylor_forward3_kernel<T>); });
  if (shape.err != cudaSuccess) return shape.err;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  // barrier words and max slots start at zero (the generation word may hold anything)
  cudaError_t e = cudaMemsetAsync(sc + adv3_ctl_offset<T>(g.C), 0, 4 * sizeof(unsigned) + 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  Geom gg = g;
  void* args[] = {&gg, (void*)&vel, (void*)&rho, (void*)&K, (void*)&thresh, (void*)&kmax, (void*)&err, (void*)&sc};
  return coop_launch(taylor_forward3_kernel<T>, shape.blocks, st, args);
}

template <class T>
cudaError_t launch_taylor_adjoint3(const Geom& g, const T* vel, const T* rho, const int* K, const double* mterm,
                                   T* mu, const T* base, T alpha, T beta, T* out, T* powers, int kmax, int* err,
                                   void* scratch, cudaStream_t st, int s_end, T* mu_m1) {
  if (kmax < 1 || kmax > kTaylorKmaxLimit || !scratch || (s_end != 0 && s_end != 1)) return cudaErrorInvalidValue;
  static std::once_flag once;
  static CoopShape shape;
  std::call_once(once, [] { shape = coop_shape(taylor_adjoint3_kernel<T>); });
  if (shape.err != cudaSuccess) return shape.err;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  cudaError_t e = cudaMemsetAsync(sc + adv3_ctl_offset<T>(g.C), 0, 4 * sizeof(unsigned) + 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  Geom gg = g;
  void* args[] = {&gg,         (void*)&vel,   (void*)&rho,  (void*)&K,   (void*)&mterm,
                  (void*)&mu,  (void*)&base,  (void*)&alpha, (void*)&beta, (void*)&out,
                  (void*)&powers, (void*)&kmax, (void*)&err, (void*)&sc, (void*)&s_end, (void*)&mu_m1};
  return coop_launch(taylor_adjoint3_kernel<T>, shape.blocks, st, args);
}

// tmp0: C doubles, tmp1: 2C doubles (used as arrays of the state type)
template <class T>
void launch_metric3(const Geom& g, const T* rho_s, const double* star, double c, int levels, double sigma0,
                    double* out, double* tmp0, double* tmp1, cudaStream_t st) {
  const int C = g.C;
  const int tpb = 256;
  const unsigned nb = (unsigned)((C + tpb - 1) / tpb);
  T* d0 = reinterpret_cast<T*>(tmp0);
  T* d1 = reinterpret_cast<T*>(tmp1);
  T* d2 = d1 + C;
  metric3_diff_kernel<T><<<nb, tpb, 0, st>>>(rho_s, star, d0, C);
  if (levels <= 0) {
    metric3_scale_kernel<T><<<nb, tpb, 0, st>>>(d0, out, c, C);
    return;
  }
  cudaMemsetAsync(out, 0, sizeof(double) * C, st);
  for (int l = 0; l < levels; ++l) {
    const double sig = sigma0 * (double)(1 << l);
    const int R = (int)ceil(3.0 * sig);
    const size_t sm = sizeof(double) * 3 * (2 * R + 1);
    const int pr = g.periodic;
    blur3_kernel<T, T><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 0, 0, sig, d0, d1, 1.0, 0, pr);       // G_x
    blur3_kernel<T, T><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 1, 0, sig, d1, d2, 1.0, 0, pr);       // G_y
    blur3_kernel<T, T><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 2, 0, sig, d2, d1, 1.0, 0, pr);       // G_z
    blur3_kernel<T, T><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 2, 1, sig, d1, d2, 1.0, 0, pr);       // G_z^T
    blur3_kernel<T, T><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 1, 1, sig, d2, d1, 1.0, 0, pr);       // G_y^T
    blur3_kernel<T, double><<<nb, tpb, sm, st>>>(g.nx, g.ny, g.nz, 0, 1, sig, d1, out, c, 1, pr);   // += c G_x^T
  }
}

#define STC_ADV3_INST(T)                                                                                        \
  template cudaError_t launch_taylor_forward3<T>(const Geom&, const T*, T*, int*, double, int, int*, void*,    \
                                                 cudaStream_t);                                                \
  template cudaError_t launch_taylor_adjoint3<T>(const Geom&, const T*, const T*, const int*, const double*,   \
                                                 T*, const T*, T, T, T*, T*, int, int*, void*, cudaStream_t,   \
                                                 int, T*);                                                     \
  template void launch_metric3<T>(const Geom&, const T*, const double*, double, int, double, double*, double*,  \
                                  double*, cudaStream_t);
STC_ADV3_INST(float)
STC_ADV3_INST(double)

}  // namespace stc
