// The forward fluid simulation with a given control u and its adjoint (the
// full-resimulation path of Sec. 5 and App. A, exposed for differentiation).
//
// One implicit step of Eq. NSA/NSB, (v - v_prev)/dt + Adv(v) - u + grad p = 0,
// div v = 0, is solved by the Picard iteration v <- Q[v_prev + dt (u - Adv(v))]
// (the projection Q supplies grad p); its linearisation's transpose by the
// transposed iteration z <- Q[y - dt dAdv(v)^T z], xi = dt z.  These kernels
// form the right-hand sides; the projections are the library's own.
#include "grid3d.cuh"
#include "stc_kernels.h"

namespace stc {
namespace {

// out = v_prev + dt (u - Adv(v)) on interior faces, 0 on walls
template <class T>
__global__ void picard_rhs_kernel(Geom g, const T* __restrict__ v_prev, const T* __restrict__ u,
                                  const T* __restrict__ v, T dt, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.F) return;
  T a = T(0);
  bool in;
  if (g.dim == 3) {
    int k, j, i;
    const int axis = g3::face_coords(g, e, k, j, i);
    in = g3::is_face(g, axis, k, j, i);
    if (in && g.self_adv) a = g3::adv(g, v, axis, k, j, i);
  } else if (e < g.Fx) {
    const int j = e / (g.nx + 1), i = e - j * (g.nx + 1);
    in = xf_interior(g, j, i);
    if (in && g.self_adv) a = adv_x(g, v, j, i);
  } else {
    const int q = e - g.Fx;
    const int j = q / g.nx, i = q - j * g.nx;
    in = yf_interior(g, j, i);
    if (in && g.self_adv) a = adv_y(g, v, j, i);
  }
  out[e] = in ? v_prev[e] + dt * (u[e] - a) : T(0);
}

// out = y - dt dAdv(v)^T z on interior faces, 0 on walls
template <class T>
__global__ void picard_adj_rhs_kernel(Geom g, const T* __restrict__ v, const T* __restrict__ y,
                                      const T* __restrict__ z, T dt, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.F) return;
  T jt = T(0);
  bool in;
  if (g.dim == 3) {
    int k, j, i;
    const int axis = g3::face_coords(g, e, k, j, i);
    in = g3::is_face(g, axis, k, j, i);
    if (in && g.self_adv) jt = g3::jtu(g, v, z, axis, k, j, i);
  } else if (e < g.Fx) {
    const int j = e / (g.nx + 1), i = e - j * (g.nx + 1);
    in = xf_interior(g, j, i);
    if (in && g.self_adv) jt = jtu_x(g, v, z, j, i);
  } else {
    const int q = e - g.Fx;
    const int j = q / g.nx, i = q - j * g.nx;
    in = yf_interior(g, j, i);
    if (in && g.self_adv) jt = jtu_y(g, v, z, j, i);
  }
  out[e] = in ? y[e] - dt * jt : T(0);
}

// out = a * x + b * y over n entries
template <class T>
__global__ void sim_axpby_kernel(size_t n, T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = a * x[e] + (y ? b * y[e] : T(0));
}

// copy with conversion and scaling between the caller's buffer and a field
template <class Ts, class Td>
__global__ void sim_copy_kernel(size_t n, const Ts* __restrict__ s, double scale, Td* d) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    d[e] = Td(scale * (double)s[e]);
}

inline unsigned blocks_of(size_t n, int tpb, unsigned cap = 8192) {
  size_t b = (n + tpb - 1) / tpb;
  if (b > cap) b = cap;
  return b == 0 ? 1u : (unsigned)b;
}

}  // namespace

template <class T>
void launch_picard_rhs(const Geom& g, const T* v_prev, const T* u, const T* v, double dt, T* out, cudaStream_t st) {
  picard_rhs_kernel<T><<<(g.F + 127) / 128, 128, 0, st>>>(g, v_prev, u, v, T(dt), out);
}

template <class T>
void launch_picard_adj_rhs(const Geom& g, const T* v, const T* y, const T* z, double dt, T* out, cudaStream_t st) {
  picard_adj_rhs_kernel<T><<<(g.F + 127) / 128, 128, 0, st>>>(g, v, y, z, T(dt), out);
}

template <class T>
void launch_sim_axpby(size_t n, double a, const T* x, double b, const T* y, T* out, cudaStream_t st) {
  if (n == 0) return;
  sim_axpby_kernel<T><<<blocks_of(n, 256), 256, 0, st>>>(n, T(a), x, T(b), y, out);
}

template <class Ts, class Td>
void launch_sim_copy(size_t n, const Ts* s, double scale, Td* d, cudaStream_t st) {
  if (n == 0) return;
  sim_copy_kernel<Ts, Td><<<blocks_of(n, 256), 256, 0, st>>>(n, s, scale, d);
}

template void launch_picard_rhs<float>(const Geom&, const float*, const float*, const float*, double, float*,
                                       cudaStream_t);
template void launch_picard_rhs<double>(const Geom&, const double*, const double*, const double*, double, double*,
                                        cudaStream_t);
template void launch_picard_adj_rhs<float>(const Geom&, const float*, const float*, const float*, double, float*,
                                           cudaStream_t);
template void launch_picard_adj_rhs<double>(const Geom&, const double*, const double*, const double*, double,
                                            double*, cudaStream_t);
template void launch_sim_axpby<float>(size_t, double, const float*, double, const float*, float*, cudaStream_t);
template void launch_sim_axpby<double>(size_t, double, const double*, double, const double*, double*, cudaStream_t);
template void launch_sim_copy<float, float>(size_t, const float*, double, float*, cudaStream_t);
template void launch_sim_copy<float, double>(size_t, const float*, double, double*, cudaStream_t);
template void launch_sim_copy<double, float>(size_t, const double*, double, float*, cudaStream_t);
template void launch_sim_copy<double, double>(size_t, const double*, double, double*, cudaStream_t);

}  // namespace stc
