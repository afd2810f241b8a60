// Solenoidal projection Q (Eq. KKTPO: the multiplier of div v* = 0 replaced by
// Q, computed with a multigrid Poisson solver, Sec. 4.1) and the elementwise
// kernels of the AO / KKT / ADMM steps.
//
// Q v = v - G phi with (D G) phi = D v on the closed box.  One CTA projects one
// face field: b = D v, phi and every coarse level live in shared memory (a
// 128^2 fp32 field needs ~171 KB; larger layouts, e.g. 128^2 in fp64, use a
// per-field scratch in global memory instead), red-black Gauss-Seidel V(2,2) cycles with
// average restriction and bilinear prolongation, the coarsest level (<= 64
// cells) by 30 parallel red-black Gauss-Seidel sweeps in fp64, then v - G phi
// written back.
#include <cmath>
#include <mutex>
#include "stc_internal.cuh"
#include "stc_kernels.h"

namespace stc {

constexpr int kPoissonThreads = 1024;
constexpr int kMaxPoissonLevels = 12;

struct PLevels {
  int n;
  int nx[kMaxPoissonLevels], ny[kMaxPoissonLevels];
  size_t off[kMaxPoissonLevels];  // element offsets of phi_l; b_l follows phi_l
};

__host__ __device__ inline PLevels poisson_levels(int nx, int ny) {
  PLevels L;
  L.n = 0;
  size_t off = 0;
  int a = nx, b = ny;
  while (true) {
    L.nx[L.n] = a;
    L.ny[L.n] = b;
    L.off[L.n] = off;
    off += 2 * (size_t)a * b;
    L.n++;
    if (L.n == kMaxPoissonLevels || a % 2 || b % 2 || a / 2 < 2 || b / 2 < 2) break;
    a /= 2;
    b /= 2;
  }
  return L;
}

__device__ __forceinline__ int ci(int n, int j, int i) { return j * n + i; }

// red-black Gauss-Seidel half sweep on level (nx, ny, h2 = h^2): phi_c = (sum phi_nb - h2 b_c)/n_nb,
// visiting only the cells of one colour (the cell of slot r in row j is
// i = 2r + ((j + colour) & 1)); dividing by 2 or 4 neighbours is a multiply
// by 1/2 or 1/4, which is exact
template <class T>
__device__ void rb_half(T* phi, const T* b, int nx, int ny, T h2, int colour) {
  const int half = (nx + 1) / 2;
  const int n = half * ny;
  RowWalk w(half);
  for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
    const int j = w.q, i = 2 * w.r + ((j + colour) & 1);
    if (i >= nx) continue;
    const int e = j * nx + i;
    T s = T(0);
    int k = 0;
    if (i > 0) { s += phi[e - 1]; ++k; }
    if (i < nx - 1) { s += phi[e + 1]; ++k; }
    if (j > 0) { s += phi[e - nx]; ++k; }
    if (j < ny - 1) { s += phi[e + nx]; ++k; }
    const T v = s - h2 * b[e];
    phi[e] = k == 4 ? v * T(0.25) : (k == 2 ? v * T(0.5) : v / T(k));
  }
}

template <class T>
__device__ __forceinline__ T lap(const T* phi, int nx, int ny, int j, int i, T ih2) {
  const int e = j * nx + i;
  T s = T(0);
  int k = 0;
  if (i > 0) { s += phi[e - 1]; ++k; }
  if (i < nx - 1) { s += phi[e + 1]; ++k; }
  if (j > 0) { s += phi[e - nx]; ++k; }
  if (j < ny - 1) { s += phi[e + nx]; ++k; }
  return (s - T(k) * phi[e]) * ih2;
}

template <class T>
__global__ void __launch_bounds__(kPoissonThreads, 1)
project_kernel(Geom g, T* fields, int vcycles, T* scratch, size_t per_field) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // all levels' phi and b: shared memory, or this field's slice of the scratch
  T* sm = scratch ? scratch + (size_t)blockIdx.x * per_field : reinterpret_cast<T*>(smem_raw);
  __shared__ double cb[64], cp[64];
  __shared__ double cmean;
  // h_l^2 and 1/h_l^2 per level, h_l = h 2^l: formed once (scaling by 4^l is
  // exact, so these equal the per-level fp64 expressions rounded to T)
  __shared__ T h2tab[16], ih2tab[16];
  const PLevels L = poisson_levels(g.nx, g.ny);
  if (threadIdx.x == 0) {
    const T h2 = T(g.h * g.h), ih2 = T(1.0 / (g.h * g.h));
    T s4 = T(1);
    for (int l = 0; l < L.n && l < 16; ++l, s4 *= T(4)) {
      h2tab[l] = h2 * s4;
      ih2tab[l] = ih2 / s4;
    }
  }
  __syncthreads();
  T* v = fields + (size_t)blockIdx.x * g.F;
  const int nx = g.nx, ny = g.ny;
  T* phi0 = sm + L.off[0];
  T* b0 = phi0 + (size_t)nx * ny;
  // b = D v, phi = 0
  {
    RowWalk w(nx);
    for (int e = threadIdx.x; e < nx * ny; e += blockDim.x, w.next()) {
      b0[e] = divergence(g, v, w.q, w.r);
      phi0[e] = T(0);
    }
  }
  __syncthreads();
  const int nl = L.n;
  for (int cyc = 0; cyc < vcycles; ++cyc) {
    // descend
    for (int l = 0; l < nl - 1; ++l) {
      const int lx = L.nx[l], ly = L.ny[l];
      const T h2 = h2tab[l], ih2 = ih2tab[l];
      T* phi = sm + L.off[l];
      T* b = phi + (size_t)lx * ly;
      if (l > 0) {
        for (int e = threadIdx.x; e < lx * ly; e += blockDim.x) phi[e] = T(0);
        __syncthreads();
      }
      for (int s = 0; s < 2; ++s) {
        rb_half(phi, b, lx, ly, h2, 0);
        __syncthreads();
        rb_half(phi, b, lx, ly, h2, 1);
        __syncthreads();
      }
      // restricted residual: b_{l+1} = mean over the 4 children of (b - L phi)
      const int cx = L.nx[l + 1], cy = L.ny[l + 1];
      T* bc = sm + L.off[l + 1] + (size_t)cx * cy;
      RowWalk wc(cx);
      for (int e = threadIdx.x; e < cx * cy; e += blockDim.x, wc.next()) {
        const int J = wc.q, I = wc.r;
        T acc = T(0);
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
          for (int di = 0; di < 2; ++di) {
            const int jj = 2 * J + dj, ii = 2 * I + di;
            acc += b[jj * lx + ii] - lap(phi, lx, ly, jj, ii, ih2);
          }
        bc[e] = T(0.25) * acc;
      }
      __syncthreads();
    }
    // coarsest (<= 64 cells): red-black Gauss-Seidel in fp64 on the compatible
    // (mean-free) right-hand side, by warp 0 alone (two cells per lane, warp
    // synchronisation between the half-sweeps)
    {
      const int l = nl - 1;
      const int lx = L.nx[l], ly = L.ny[l];
      const int n = lx * ly;
      const double h2 = (g.h * (double)(1 << l)) * (g.h * (double)(1 << l));
      T* phi = sm + L.off[l];
      T* b = phi + (size_t)n;
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int e = lane; e < n; e += 32) {
          cb[e] = (double)b[e];
          cp[e] = 0.0;
        }
        __syncwarp();
        if (lane == 0) {
          double m = 0.0;
          for (int k = 0; k < n; ++k) m += cb[k];
          cmean = m / n;
        }
        __syncwarp();
        for (int e = lane; e < n; e += 32) cb[e] -= cmean;
        __syncwarp();
        // a lane's (up to) two cells, their neighbour counts and reciprocals
        int ce[2], cc[2];
        double ikn[2];
        for (int q = 0; q < 2; ++q) {
          const int e = lane + 32 * q;
          ce[q] = e;
          const int j = e / lx, i = e - (e / lx) * lx;
          cc[q] = (i + j) & 1;
          const int kn = (i > 0) + (i < lx - 1) + (j > 0) + (j < ly - 1);
          ikn[q] = kn > 0 ? 1.0 / kn : 0.0;
        }
        for (int it = 0; it < 30; ++it)
          for (int colour = 0; colour < 2; ++colour) {
            for (int q = 0; q < 2; ++q) {
              const int e = ce[q];
              if (e < n && cc[q] == colour) {
                const int j = e / lx, i = e - (e / lx) * lx;
                double sacc = 0.0;
                if (i > 0) sacc += cp[e - 1];
                if (i < lx - 1) sacc += cp[e + 1];
                if (j > 0) sacc += cp[e - lx];
                if (j < ly - 1) sacc += cp[e + lx];
                cp[e] = (sacc - h2 * cb[e]) * ikn[q];
              }
            }
            __syncwarp();
          }
        for (int e = lane; e < n; e += 32) phi[e] = T(cp[e]);
      }
      __syncthreads();
    }
    // ascend: phi_l += P phi_{l+1}, post-smooth
    for (int l = nl - 2; l >= 0; --l) {
      const int lx = L.nx[l], ly = L.ny[l];
      const int cx = L.nx[l + 1], cy = L.ny[l + 1];
      const T h2 = h2tab[l];
      T* phi = sm + L.off[l];
      T* b = phi + (size_t)lx * ly;
      const T* pc = sm + L.off[l + 1];
      RowWalk wf(lx);
      for (int e = threadIdx.x; e < lx * ly; e += blockDim.x, wf.next()) {
        const int j = wf.q, i = wf.r;
        const int ja = j >> 1, ia = i >> 1;
        int jb = (j & 1) ? ja + 1 : ja - 1;
        int ib = (i & 1) ? ia + 1 : ia - 1;
        jb = jb < 0 ? 0 : (jb > cy - 1 ? cy - 1 : jb);
        ib = ib < 0 ? 0 : (ib > cx - 1 ? cx - 1 : ib);
        phi[e] += T(0.5625) * pc[ja * cx + ia] + T(0.1875) * pc[ja * cx + ib] + T(0.1875) * pc[jb * cx + ia] +
                  T(0.0625) * pc[jb * cx + ib];
      }
      __syncthreads();
      for (int s = 0; s < 2; ++s) {
        rb_half(phi, b, lx, ly, h2, 0);
        __syncthreads();
        rb_half(phi, b, lx, ly, h2, 1);
        __syncthreads();
      }
    }
  }
  // v -= G phi on interior faces
  for (int e = threadIdx.x; e < g.F; e += blockDim.x) {
    if (e < g.Fx) {
      const int j = e / (nx + 1), i = e - j * (nx + 1);
      if (i >= 1 && i <= nx - 1) v[e] -= (phi0[j * nx + i] - phi0[j * nx + i - 1]) * pick<T>(g.ih, g.ihf);
      else v[e] = T(0);
    } else {
      const int q = e - g.Fx;
      const int j = q / nx, i = q - j * nx;
      if (j >= 1 && j <= ny - 1) v[e] -= (phi0[j * nx + i] - phi0[(j - 1) * nx + i]) * pick<T>(g.ih, g.ihf);
      else v[e] = T(0);
    }
  }
}

size_t project_smem(const Geom& g, size_t tsize) {
  const PLevels L = poisson_levels(g.nx, g.ny);
  const int l = L.n - 1;
  return (L.off[l] + 2 * (size_t)L.nx[l] * L.ny[l]) * tsize;
}

bool project_supported(const Geom& g, size_t) {
  const PLevels L = poisson_levels(g.nx, g.ny);
  const int l = L.n - 1;
  return L.nx[l] * L.ny[l] <= 64;   // the coarsest solve's fp64 arrays
}

bool project_needs_scratch(const Geom& g, size_t tsize) { return project_smem(g, tsize) > kProjectSmemLimit; }

// ---------------------------------------------------------------------------
// Exact Q on the closed 2D box.  The cell-centred Neumann Laplacian D G of the
// uniform grid is diagonalised by the orthonormal DCT-II in each axis:
// D G = (C_y (x) C_x)^T diag(lam) (C_y (x) C_x), C[k][i] = s_k cos(pi k (2i+1) / 2n),
// lam = -(4/h^2) (sin^2(pi kx / 2nx) + sin^2(pi ky / 2ny)).  So
// phi = C_y^T [(C_y b C_x^T) / lam] C_x, with 1/lam_00 = 0 dropping the
// constant (the null space, which G removes anyway): four dense products per
// field.  One CTA per field, b and the intermediates in shared memory, 4x4
// outputs per thread.  This is Q itself to rounding, where the multigrid gives
// Q to its truncation after `vcycles` cycles.
// ---------------------------------------------------------------------------
size_t project_dct_elems(const Geom& g) {
  return 2 * (size_t)g.nx * g.nx + 2 * (size_t)g.ny * g.ny + (size_t)g.nx * g.ny;
}

bool project_dct_fits(const Geom& g, size_t tsize) {
  return g.dim == 2 && 2 * (size_t)g.nx * g.ny * tsize <= kProjectSmemLimit;
}

// C_x, C_x^T, C_y, C_y^T, 1/lam (row ky, column kx), in fp64
void project_dct_tables(const Geom& g, double* out) {
  const double pi = 3.14159265358979323846;
  auto basis = [&](int n, double* C, double* CT) {
    for (int k = 0; k < n; ++k) {
      const double sk = std::sqrt((k == 0 ? 1.0 : 2.0) / n);
      for (int i = 0; i < n; ++i) {
        const double c = sk * std::cos(pi * k * (2.0 * i + 1.0) / (2.0 * n));
        C[(size_t)k * n + i] = c;
        CT[(size_t)i * n + k] = c;
      }
    }
  };
  double* Cx = out;
  double* CxT = Cx + (size_t)g.nx * g.nx;
  double* Cy = CxT + (size_t)g.nx * g.nx;
  double* CyT = Cy + (size_t)g.ny * g.ny;
  double* il = CyT + (size_t)g.ny * g.ny;
  basis(g.nx, Cx, CxT);
  basis(g.ny, Cy, CyT);
  const double ih2 = 1.0 / (g.h * g.h);
  for (int ky = 0; ky < g.ny; ++ky)
    for (int kx = 0; kx < g.nx; ++kx) {
      const double sx = std::sin(pi * kx / (2.0 * g.nx)), sy = std::sin(pi * ky / (2.0 * g.ny));
      const double lam = -4.0 * ih2 * (sx * sx + sy * sy);
      il[(size_t)ky * g.nx + kx] = (kx == 0 && ky == 0) ? 0.0 : 1.0 / lam;
    }
}

// out[r][c] = (sum_k A[r][k] B[k][c]) * (scale ? scale[r][c] : 1), all row-major
// (leading dimensions lda, ldb, Cc); k in order, so the result is deterministic
template <class T>
__device__ __forceinline__ void dct_gemm(T* out, const T* A, int lda, const T* B, int ldb, int R, int Cc, int K,
                                         const T* __restrict__ scale) {
  const int ntr = (R + 3) >> 2, ntc = (Cc + 3) >> 2;
  const bool vec = (Cc & 3) == 0 && (ldb & 3) == 0;
  for (int t = threadIdx.x; t < ntr * ntc; t += blockDim.x) {
    const int r0 = (t / ntc) * 4, c0 = (t - (t / ntc) * ntc) * 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k = 0; k < K; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = r0 + i < R ? A[(size_t)(r0 + i) * lda + k] : T(0);
      const T* bk = B + (size_t)k * ldb + c0;
      if (vec) {
        if constexpr (sizeof(T) == 4) {
          const float4 q = *reinterpret_cast<const float4*>(bk);
          b[0] = q.x;
          b[1] = q.y;
          b[2] = q.z;
          b[3] = q.w;
        } else {
          const double2 q0 = reinterpret_cast<const double2*>(bk)[0], q1 = reinterpret_cast<const double2*>(bk)[1];
          b[0] = q0.x;
          b[1] = q0.y;
          b[2] = q1.x;
          b[3] = q1.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = c0 + j < Cc ? bk[j] : T(0);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (r0 + i < R && c0 + j < Cc) {
          const size_t e = (size_t)(r0 + i) * Cc + c0 + j;
          out[e] = scale ? acc[i][j] * scale[e] : acc[i][j];
        }
  }
}

template <class T>
__global__ void __launch_bounds__(kPoissonThreads, 1)
project_dct_kernel(Geom g, T* fields, const T* __restrict__ tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = g.nx, ny = g.ny;
  T* S1 = reinterpret_cast<T*>(smem_raw);             // [ny][nx]
  T* S2 = S1 + (size_t)nx * ny;                       // [ny][nx]
  const T* Cx = tab;
  const T* CxT = Cx + (size_t)nx * nx;
  const T* Cy = CxT + (size_t)nx * nx;
  const T* CyT = Cy + (size_t)ny * ny;
  const T* il = CyT + (size_t)ny * ny;
  T* v = fields + (size_t)blockIdx.x * g.F;
  {
    RowWalk w(nx);
    for (int e = threadIdx.x; e < nx * ny; e += blockDim.x, w.next()) S1[e] = divergence(g, v, w.q, w.r);
  }
  __syncthreads();
  dct_gemm(S2, Cy, ny, S1, nx, ny, nx, ny, (const T*)nullptr);   // C_y b
  __syncthreads();
  dct_gemm(S1, S2, nx, CxT, nx, ny, nx, nx, il);                 // (C_y b C_x^T) / lam
  __syncthreads();
  dct_gemm(S2, CyT, ny, S1, nx, ny, nx, ny, (const T*)nullptr);  // C_y^T (.)
  __syncthreads();
  dct_gemm(S1, S2, nx, Cx, nx, ny, nx, nx, (const T*)nullptr);   // (.) C_x = phi
  __syncthreads();
  const T ih = pick<T>(g.ih, g.ihf);
  for (int e = threadIdx.x; e < g.F; e += blockDim.x) {
    if (e < g.Fx) {
      const int j = e / (nx + 1), i = e - j * (nx + 1);
      if (i >= 1 && i <= nx - 1) v[e] -= (S1[j * nx + i] - S1[j * nx + i - 1]) * ih;
      else v[e] = T(0);
    } else {
      const int q = e - g.Fx;
      const int j = q / nx, i = q - j * nx;
      if (j >= 1 && j <= ny - 1) v[e] -= (S1[j * nx + i] - S1[(j - 1) * nx + i]) * ih;
      else v[e] = T(0);
    }
  }
}

template <class T>
static cudaError_t launch_project_dct(const Geom& g, T* fields, int count, cudaStream_t st, const T* tab) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (attr_err == cudaSuccess) attr_err = cudaFuncGetAttributes(&fa, (const void*)project_dct_kernel<T>);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute((const void*)project_dct_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin - (int)fa.sharedSizeBytes);
  });
  if (attr_err != cudaSuccess) return attr_err;
  project_dct_kernel<T><<<count, kPoissonThreads, 2 * (size_t)g.nx * g.ny * sizeof(T), st>>>(g, fields, tab);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_project(const Geom& g, T* fields, int count, int vcycles, cudaStream_t st, T* scratch,
                           const T* dct) {
  if (g.dim == 3) return launch_project3<T>(g, fields, count, vcycles, st, scratch);
  if (count <= 0) return cudaSuccess;
  if (dct && project_dct_fits(g, sizeof(T))) return launch_project_dct<T>(g, fields, count, st, dct);
  const size_t layout = project_smem(g, sizeof(T));
  if (project_needs_scratch(g, sizeof(T)) && !scratch) return cudaErrorInvalidValue;
  const size_t sm = scratch ? 0 : layout;
  // raise the cap once to the opt-in maximum (per-size settings would race
  // between host threads solving problems of different sizes)
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (attr_err == cudaSuccess) attr_err = cudaFuncGetAttributes(&fa, (const void*)project_kernel<T>);
    // the cap covers dynamic memory only: opt-in total minus the static arrays
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute((const void*)project_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin - (int)fa.sharedSizeBytes);
  });
  if (attr_err != cudaSuccess) return attr_err;
  project_kernel<T><<<count, kPoissonThreads, sm, st>>>(g, fields, vcycles, scratch, layout / sizeof(T));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
// w_s = v_s + lambda_s / K (s >= 1), w_0 = v_0; v*_s = w_s unless warm-starting
// (Alg. 1 initialisation; v*_0 = v_0 always)
template <class T>
__global__ void ao_init_kernel(Geom g, const T* __restrict__ v, const T* __restrict__ lam, double invK, T* w,
                               T* vstar, int warm) {
  const size_t n = (size_t)g.N * g.F;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    T val = v[e];
    if (e >= (size_t)g.F) val += T(invK) * lam[e];
    w[e] = val;
    if (!warm || e < (size_t)g.F) vstar[e] = val;
  }
}

template <class T>
__global__ void axpby_kernel(size_t n, const T* __restrict__ a, double alpha, const T* __restrict__ b, double beta,
                             T* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = T(alpha) * a[e] + T(beta) * b[e];
}

// u_raw_t = (v_{t+1} - v_t)/dt + Adv(v_{t+1}), t = 0..N-1   (Appendix A)
template <class T>
__global__ void kkt_force_rhs_kernel(Geom g, const T* __restrict__ v, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (e >= g.F || t >= g.N) return;
  const T* vn = v + (size_t)(t + 1) * g.F;
  const T* vt = v + (size_t)t * g.F;
  T val = T(0);
  if (e < g.Fx) {
    const int j = e / (g.nx + 1), i = e - j * (g.nx + 1);
    if (xf_interior(g, j, i)) val = (vn[e] - vt[e]) * pick<T>(g.idt, g.idtf) + T(g.self_adv) * adv_x(g, vn, j, i);
  } else {
    const int q = e - g.Fx;
    const int j = q / g.nx, i = q - j * g.nx;
    if (yf_interior(g, j, i)) val = (vn[e] - vt[e]) * pick<T>(g.idt, g.idtf) + T(g.self_adv) * adv_y(g, vn, j, i);
  }
  out[(size_t)t * g.F + e] = val;
}

// g_raw_t = r(u_{t-1}/dt + dAdv(v_t)^T u_{t-1} - u_t/dt [t<N]) + dens_t, t = 1..N
template <class T>
__global__ void kkt_grad_rhs_kernel(Geom g, const T* __restrict__ v, const T* __restrict__ u,
                                    const T* __restrict__ dens, double r, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y + 1;
  if (e >= g.F || t > g.N) return;
  const T* vt = v + (size_t)t * g.F;
  const T* um = u + (size_t)(t - 1) * g.F;
  T val = T(0);
  bool inter;
  T jt = T(0);
  if (e < g.Fx) {
    const int j = e / (g.nx + 1), i = e - j * (g.nx + 1);
    inter = xf_interior(g, j, i);
    if (inter && g.self_adv) jt = jtu_x(g, vt, um, j, i);
  } else {
    const int q = e - g.Fx;
    const int j = q / g.nx, i = q - j * g.nx;
    inter = yf_interior(g, j, i);
    if (inter && g.self_adv) jt = jtu_y(g, vt, um, j, i);
  }
  if (inter) {
    T s = um[e] * pick<T>(g.idt, g.idtf) + jt;
    if (t < g.N) s -= u[(size_t)t * g.F + e] * pick<T>(g.idt, g.idtf);
    val = T(r) * s + dens[(size_t)t * g.F + e];
  }
  out[(size_t)t * g.F + e] = val;
}

__device__ __forceinline__ void atomic_max_nonneg2(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class T>
__global__ void absdiff_max_copy_kernel(const T* __restrict__ a, T* b, size_t n, double* out) {
  double m = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    m = fmax(m, fabs((double)a[e] - (double)b[e]));
    b[e] = a[e];
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg2(out, m);
}

// AO blend (Sec. 5): out = x + a (y - x); a blend of solenoidal fields is solenoidal
template <class T>
__global__ void blend_kernel(size_t n, const T* __restrict__ x, const T* __restrict__ y, double a, T* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = x[e] + T(a) * (y[e] - x[e]);
}


// keyframe misfit of Eq. opt in the C_i metric: 0.5 (rho - rho*)^T m with m = C (rho - rho*)
template <class T>
__global__ void misfit_dot_kernel(int C, const T* __restrict__ rho, const double* __restrict__ star,
                                  const double* __restrict__ m, double* out, RedScratch rs) {
  double s = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C; e += gridDim.x * blockDim.x)
    s += ((double)rho[e] - star[e]) * m[e];
  block_sum_ordered(0.5 * s, out, rs);
}

template <class T>
__global__ void diff_sumsq_kernel(size_t n, const T* __restrict__ a, const T* __restrict__ b, double scale,
                                  double* out, RedScratch rs) {
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double d = (double)a[e] - (double)b[e];
    s += d * d;
  }
  block_sum_ordered(scale * s, out, rs);
}

static inline unsigned nblk(size_t n, int tpb, unsigned cap = 4096) {
  size_t b = (n + tpb - 1) / tpb;
  if (b > cap) b = cap;
  return b == 0 ? 1u : (unsigned)b;
}

template <class T>
void launch_ao_init(const Geom& g, const T* v, const T* lam, double invK, T* w, T* vstar, int warm,
                    cudaStream_t st) {
  ao_init_kernel<T><<<nblk((size_t)g.N * g.F, 256), 256, 0, st>>>(g, v, lam, invK, w, vstar, warm);
}
template <class T>
void launch_axpby_faces(const Geom& g, int count, const T* a, double alpha, const T* b, double beta, T* out,
                        cudaStream_t st) {
  const size_t n = (size_t)count * g.F;
  if (n == 0) return;
  axpby_kernel<T><<<nblk(n, 256), 256, 0, st>>>(n, a, alpha, b, beta, out);
}
template <class T>
void launch_kkt_force_rhs(const Geom& g, const T* v, T* out, cudaStream_t st) {
  if (g.dim == 3) return launch_kkt_force_rhs3<T>(g, v, out, st);
  dim3 grid((g.F + 127) / 128, g.N);
  kkt_force_rhs_kernel<T><<<grid, 128, 0, st>>>(g, v, out);
}
template <class T>
void launch_kkt_grad_rhs(const Geom& g, const T* v, const T* u, const T* dens, double r, T* out, cudaStream_t st) {
  if (g.dim == 3) return launch_kkt_grad_rhs3<T>(g, v, u, dens, r, out, st);
  dim3 grid((g.F + 127) / 128, g.N);
  kkt_grad_rhs_kernel<T><<<grid, 128, 0, st>>>(g, v, u, dens, r, out);
}
template <class T>
void launch_absdiff_max_copy(const T* a, T* b, size_t n, double* out, cudaStream_t st) {
  absdiff_max_copy_kernel<T><<<nblk(n, 256, 1216), 256, 0, st>>>(a, b, n, out);
}

template <class T>
void launch_blend_faces(const Geom& g, int count, const T* x, const T* y, double a, T* out, cudaStream_t st) {
  const size_t n = (size_t)count * g.F;
  if (n == 0) return;
  blend_kernel<T><<<nblk(n, 256), 256, 0, st>>>(n, x, y, a, out);
}
template <class T>
void launch_misfit_dot(const Geom& g, const T* rho, const double* star, const double* m, double* out,
                       cudaStream_t st, RedScratch rs) {
  misfit_dot_kernel<T><<<nblk(g.C, 256, 304), 256, 0, st>>>(g.C, rho, star, m, out, rs);
}
template <class T>
void launch_diff_sumsq(const T* a, const T* b, size_t n, double scale, double* out, cudaStream_t st,
                       RedScratch rs) {
  if (n == 0) return;
  diff_sumsq_kernel<T><<<nblk(n, 256, kReduceMaxBlocks), 256, 0, st>>>(n, a, b, scale, out, rs);
}

#define STC_POI_INST(T)                                                                                        \
  template cudaError_t launch_project<T>(const Geom&, T*, int, int, cudaStream_t, T*, const T*);              \
  template void launch_ao_init<T>(const Geom&, const T*, const T*, double, T*, T*, int, cudaStream_t);             \
  template void launch_axpby_faces<T>(const Geom&, int, const T*, double, const T*, double, T*, cudaStream_t); \
  template void launch_kkt_force_rhs<T>(const Geom&, const T*, T*, cudaStream_t);                             \
  template void launch_kkt_grad_rhs<T>(const Geom&, const T*, const T*, const T*, double, T*, cudaStream_t);  \
  template void launch_absdiff_max_copy<T>(const T*, T*, size_t, double*, cudaStream_t);                   \
  template void launch_blend_faces<T>(const Geom&, int, const T*, const T*, double, T*, cudaStream_t);        \
  template void launch_misfit_dot<T>(const Geom&, const T*, const double*, const double*, double*,            \
                                     cudaStream_t, RedScratch);                                               \
  template void launch_diff_sumsq<T>(const T*, const T*, size_t, double, double*, cudaStream_t, RedScratch);
STC_POI_INST(float)
STC_POI_INST(double)

}  // namespace stc
