// Solenoidal projection Q on the 3D grid (Eq. KKTPO; the multigrid Poisson
// solve of Sec. 4.1): Q v = v - G phi with (D G) phi = D v on the closed box.
//
// A 3D field does not fit one CTA's shared memory, so all `count` fields of a
// call are solved together by a multigrid over global memory: every kernel
// below runs over (field, cell) pairs of one level, so each launch fills the
// GPU.  Red-black Gauss-Seidel V(2,2) cycles, residual restriction by the
// mean of the 8 children, trilinear prolongation, the coarsest level (<= 512
// cells) by 60 red-black sweeps in fp64 in shared memory (one CTA per field,
// on the mean-free right-hand side) -- the same cycle as the 2D on-chip solver.
#include "grid3d.cuh"
#include "stc_kernels.h"

namespace stc {
namespace {

using namespace g3;

constexpr int kMaxP3Levels = 12;
constexpr int kCoarsestMaxCells = 512;

struct P3Levels {
  int n;
  int nx[kMaxP3Levels], ny[kMaxP3Levels], nz[kMaxP3Levels];
  size_t off[kMaxP3Levels];   // element offset of level l's phi (count x C_l); b_l follows it
  size_t total;               // elements of all levels
};

P3Levels p3_levels(const Geom& g, int count) {
  P3Levels L;
  L.n = 0;
  size_t off = 0;
  int a = g.nx, b = g.ny, c = g.nz;
  while (true) {
    L.nx[L.n] = a;
    L.ny[L.n] = b;
    L.nz[L.n] = c;
    L.off[L.n] = off;
    off += 2 * (size_t)count * a * b * c;
    L.n++;
    if (L.n == kMaxP3Levels || a % 2 || b % 2 || c % 2 || a / 2 < 2 || b / 2 < 2 || c / 2 < 2) break;
    a /= 2;
    b /= 2;
    c /= 2;
  }
  L.total = off;
  return L;
}

struct Lv {
  int nx, ny, nz, C;
  int periodic;   // neighbours wrap (no walls: 6 neighbours everywhere)
};

// neighbour sum and count of cell (k, j, i) on a level
template <class Acc>
__device__ __forceinline__ int p3_neighbours(const Lv& L, int k, int j, int i, Acc acc) {
  if (L.periodic) {
    const int im = i > 0 ? i - 1 : L.nx - 1, ip = i < L.nx - 1 ? i + 1 : 0;
    const int jm = j > 0 ? j - 1 : L.ny - 1, jp = j < L.ny - 1 ? j + 1 : 0;
    const int km = k > 0 ? k - 1 : L.nz - 1, kp = k < L.nz - 1 ? k + 1 : 0;
    acc((k * L.ny + j) * L.nx + im);
    acc((k * L.ny + j) * L.nx + ip);
    acc((k * L.ny + jm) * L.nx + i);
    acc((k * L.ny + jp) * L.nx + i);
    acc((km * L.ny + j) * L.nx + i);
    acc((kp * L.ny + j) * L.nx + i);
    return 6;
  }
  const int c = (k * L.ny + j) * L.nx + i;
  int nn = 0;
  if (i > 0) { acc(c - 1); ++nn; }
  if (i < L.nx - 1) { acc(c + 1); ++nn; }
  if (j > 0) { acc(c - L.nx); ++nn; }
  if (j < L.ny - 1) { acc(c + L.nx); ++nn; }
  if (k > 0) { acc(c - L.nx * L.ny); ++nn; }
  if (k < L.nz - 1) { acc(c + L.nx * L.ny); ++nn; }
  return nn;
}

template <class T>
__global__ void p3_div_kernel(Geom g, const T* __restrict__ fields, int count, T* phi, T* b) {
  const size_t n = (size_t)count * g.C;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / g.C), c = (int)(e - (size_t)f * g.C);
    const int i = c % g.nx, r = c / g.nx, j = r % g.ny, k = r / g.ny;
    b[e] = divergence(g, fields + (size_t)f * g.F, k, j, i);
    phi[e] = T(0);
  }
}

// one colour of red-black Gauss-Seidel: phi_c = (sum phi_nb - h2 b_c) / n_nb
template <class T>
__global__ void p3_rb_kernel(Lv L, int count, T* phi, const T* __restrict__ b, T h2, int colour) {
  const int half = (L.nx + 1) / 2;
  const size_t rows = (size_t)L.ny * L.nz;
  const size_t n = (size_t)count * rows * half;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int slot = (int)(e % half);
    const size_t rr = e / half;
    const int row = (int)(rr % rows);
    const int f = (int)(rr / rows);
    const int j = row % L.ny, k = row / L.ny;
    const int i = 2 * slot + ((j + k + colour) & 1);
    if (i >= L.nx) continue;
    T* p = phi + (size_t)f * L.C;
    const int c = (k * L.ny + j) * L.nx + i;
    T s = T(0);
    const int nn = p3_neighbours(L, k, j, i, [&](int q) { s += p[q]; });
    p[c] = (s - h2 * b[(size_t)f * L.C + c]) / T(nn);
  }
}

template <class T>
__device__ __forceinline__ T p3_lap(const T* p, Lv L, int k, int j, int i, T ih2) {
  const int c = (k * L.ny + j) * L.nx + i;
  T s = T(0);
  const int nn = p3_neighbours(L, k, j, i, [&](int q) { s += p[q]; });
  return (s - T(nn) * p[c]) * ih2;
}

// b_{l+1} = mean over the 8 children of (b - L phi); phi_{l+1} = 0
template <class T>
__global__ void p3_restrict_kernel(Lv F, Lv Cc, int count, const T* __restrict__ phi, const T* __restrict__ b,
                                   T* phic, T* bc, T ih2) {
  const size_t n = (size_t)count * Cc.C;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / Cc.C), c = (int)(e - (size_t)f * Cc.C);
    const int I = c % Cc.nx, r = c / Cc.nx, J = r % Cc.ny, K = r / Cc.ny;
    const T* p = phi + (size_t)f * F.C;
    const T* bb = b + (size_t)f * F.C;
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int k = 2 * K + a, j = 2 * J + d, i = 2 * I + q;
          acc += bb[(k * F.ny + j) * F.nx + i] - p3_lap(p, F, k, j, i, ih2);
        }
    bc[e] = T(0.125) * acc;
    phic[e] = T(0);
  }
}

__device__ __forceinline__ void p3_interp(int k, int nc, int& a, int& b, bool periodic) {
  a = k >> 1;
  b = (k & 1) ? a + 1 : a - 1;
  if (periodic) b = b < 0 ? b + nc : (b > nc - 1 ? b - nc : b);
  else b = b < 0 ? 0 : (b > nc - 1 ? nc - 1 : b);
}

// phi_l += P phi_{l+1} (trilinear, (3/4, 1/4) per axis, clamped)
template <class T>
__global__ void p3_prolong_kernel(Lv F, Lv Cc, int count, T* phi, const T* __restrict__ phic) {
  const size_t n = (size_t)count * F.C;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / F.C), c = (int)(e - (size_t)f * F.C);
    const int i = c % F.nx, r = c / F.nx, j = r % F.ny, k = r / F.ny;
    int ka, kb, ja, jb, ia, ib;
    p3_interp(k, Cc.nz, ka, kb, F.periodic != 0);
    p3_interp(j, Cc.ny, ja, jb, F.periodic != 0);
    p3_interp(i, Cc.nx, ia, ib, F.periodic != 0);
    const T* pc = phic + (size_t)f * Cc.C;
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const T w = (a ? T(0.25) : T(0.75)) * (d ? T(0.25) : T(0.75)) * (q ? T(0.25) : T(0.75));
          acc += w * pc[((a ? kb : ka) * Cc.ny + (d ? jb : ja)) * Cc.nx + (q ? ib : ia)];
        }
    phi[e] += acc;
  }
}

// coarsest level: one CTA per field, fp64 red-black sweeps on the mean-free rhs
template <class T>
__global__ void p3_coarsest_kernel(Lv L, T* phi, const T* __restrict__ b, double h2, int sweeps) {
  __shared__ double cb[kCoarsestMaxCells], cp[kCoarsestMaxCells];
  __shared__ double mean;
  const int f = blockIdx.x;
  const int n = L.C;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    cb[e] = (double)b[(size_t)f * n + e];
    cp[e] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int e = 0; e < n; ++e) m += cb[e];
    mean = m / n;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) cb[e] -= mean;
  __syncthreads();
  for (int it = 0; it < sweeps; ++it)
    for (int colour = 0; colour < 2; ++colour) {
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e % L.nx, r = e / L.nx, j = r % L.ny, k = r / L.ny;
        if (((i + j + k) & 1) != colour) continue;
        double s = 0.0;
        const int nn = p3_neighbours(L, k, j, i, [&](int q) { s += cp[q]; });
        cp[e] = nn > 0 ? (s - h2 * cb[e]) / nn : 0.0;
      }
      __syncthreads();
    }
  for (int e = threadIdx.x; e < n; e += blockDim.x) phi[(size_t)f * n + e] = T(cp[e]);
}

// v -= G phi on interior faces, 0 on walls
template <class T>
__global__ void p3_grad_sub_kernel(Geom g, T* fields, int count, const T* __restrict__ phi) {
  const size_t n = (size_t)count * g.F;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int fi = (int)(e / g.F), f = (int)(e - (size_t)fi * g.F);
    int k, j, i;
    const int axis = face_coords(g, f, k, j, i);
    T* v = fields + (size_t)fi * g.F;
    if (is_face(g, axis, k, j, i)) v[f] -= grad(g, phi + (size_t)fi * g.C, axis, k, j, i);
    else v[f] = T(0);
  }
}

inline unsigned nb3(size_t n, int tpb) {
  size_t b = (n + tpb - 1) / tpb;
  if (b > 65535u * 8) b = 65535u * 8;
  return b == 0 ? 1u : (unsigned)b;
}

}  // namespace

size_t project3_scratch_elems(const Geom& g, int count) { return p3_levels(g, count).total; }

bool project3_supported(const Geom& g) {
  const P3Levels L = p3_levels(g, 1);
  const int l = L.n - 1;
  return (size_t)L.nx[l] * L.ny[l] * L.nz[l] <= (size_t)kCoarsestMaxCells;
}

template <class T>
cudaError_t launch_project3(const Geom& g, T* fields, int count, int vcycles, cudaStream_t st, T* scratch) {
  if (count <= 0) return cudaSuccess;
  if (!scratch || !project3_supported(g)) return cudaErrorInvalidValue;
  const P3Levels P = p3_levels(g, count);
  const int tpb = 256;
  auto lv = [&](int l) {
    Lv L;
    L.nx = P.nx[l];
    L.ny = P.ny[l];
    L.nz = P.nz[l];
    L.C = L.nx * L.ny * L.nz;
    L.periodic = g.periodic;
    return L;
  };
  auto phi_of = [&](int l) { return scratch + P.off[l]; };
  auto b_of = [&](int l) { return scratch + P.off[l] + (size_t)count * lv(l).C; };
  // h_l^2 = (h 2^l)^2 (powers of 4 exact in any precision)
  auto h2 = [&](int l) { return g.h * g.h * (double)(1u << (2 * l)); };
  p3_div_kernel<T><<<nb3((size_t)count * g.C, tpb), tpb, 0, st>>>(g, fields, count, phi_of(0), b_of(0));
  const int nl = P.n;
  for (int cyc = 0; cyc < vcycles; ++cyc) {
    for (int l = 0; l < nl - 1; ++l) {
      const Lv L = lv(l), Cc = lv(l + 1);
      const size_t nh = (size_t)count * L.ny * L.nz * ((L.nx + 1) / 2);
      for (int s = 0; s < 2; ++s)
        for (int colour = 0; colour < 2; ++colour)
          p3_rb_kernel<T><<<nb3(nh, tpb), tpb, 0, st>>>(L, count, phi_of(l), b_of(l), T(h2(l)), colour);
      p3_restrict_kernel<T><<<nb3((size_t)count * Cc.C, tpb), tpb, 0, st>>>(L, Cc, count, phi_of(l), b_of(l),
                                                                            phi_of(l + 1), b_of(l + 1),
                                                                            T(1.0 / h2(l)));
    }
    {
      const Lv L = lv(nl - 1);
      p3_coarsest_kernel<T><<<count, 256, 0, st>>>(L, phi_of(nl - 1), b_of(nl - 1), h2(nl - 1), 60);
    }
    for (int l = nl - 2; l >= 0; --l) {
      const Lv L = lv(l), Cc = lv(l + 1);
      p3_prolong_kernel<T><<<nb3((size_t)count * L.C, tpb), tpb, 0, st>>>(L, Cc, count, phi_of(l), phi_of(l + 1));
      const size_t nh = (size_t)count * L.ny * L.nz * ((L.nx + 1) / 2);
      for (int s = 0; s < 2; ++s)
        for (int colour = 0; colour < 2; ++colour)
          p3_rb_kernel<T><<<nb3(nh, tpb), tpb, 0, st>>>(L, count, phi_of(l), b_of(l), T(h2(l)), colour);
    }
  }
  p3_grad_sub_kernel<T><<<nb3((size_t)count * g.F, tpb), tpb, 0, st>>>(g, fields, count, phi_of(0));
  return cudaGetLastError();
}

// launches of one launch_project3 call (for launch accounting)
int project3_launches(const Geom& g, int vcycles) {
  const P3Levels P = p3_levels(g, 1);
  return 2 + vcycles * (10 * (P.n - 1) + 1);
}

template cudaError_t launch_project3<float>(const Geom&, float*, int, int, cudaStream_t, float*);
template cudaError_t launch_project3<double>(const Geom&, double*, int, int, cudaStream_t, double*);

}  // namespace stc
