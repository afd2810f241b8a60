// 3D staggered-grid helpers of libstc (Sec. 3.1 on an nx x ny x nz grid).
//
// Layout: cells (k, j, i), i fastest; a face field holds the x-faces
// [nz][ny][nx+1], then the y-faces [nz][ny+1][nx], then the z-faces
// [nz+1][ny][nx]; wall faces are stored and always hold 0 (closed box).
// Vorticity components live on edges: omega_x on x-edges ((i+1/2)h, jh, kh),
// omega_y on y-edges (ih, (j+1/2)h, kh), omega_z on z-edges (ih, jh, (k+1/2)h);
// an edge lying in a wall carries 0 (free slip, as the nodes of the 2D grid).
//
// Self-advection Adv[v] = (curl v) x v (Eq. NSA) at an interior a-face:
//   Adv_a = O1 * V1 - O2 * V2,
//   O1 = mean of the two omega_{a+1} edges on the face, V1 = mean of the four
//        v_{a+2} faces around it; O2, V2 likewise with a+2 and a+1
// (axes cyclic: x -> y -> z -> x).  On a field that does not vary along one
// axis and has no velocity along it, this is the 2D operator of the other two.
//
// Periodic grids (Geom::periodic): every neighbour index wraps modulo the axis
// length, so there are no walls; the layout keeps n + 1 face slots per axis
// and slot n is not a face (held at zero).  Index helpers take the cell or
// face coordinate with offsets of at most +-2 and wrap them; `interior`
// answers for neighbours (always true when periodic), `is_face` for
// coordinates decoded from a slot (false only for the unused slot n).
#pragma once

#include "stc_internal.cuh"

namespace stc {
namespace g3 {

// wrap a coordinate with |offset| <= n into [0, n) on a periodic grid
__host__ __device__ __forceinline__ int wr(const Geom& g, int a, int n) {
  return g.periodic ? (a < 0 ? a + n : (a >= n ? a - n : a)) : a;
}

__host__ __device__ __forceinline__ int xf(const Geom& g, int k, int j, int i) {
  return (wr(g, k, g.nz) * g.ny + wr(g, j, g.ny)) * (g.nx + 1) + wr(g, i, g.nx);
}
__host__ __device__ __forceinline__ int yf(const Geom& g, int k, int j, int i) {
  return g.Fx + (wr(g, k, g.nz) * (g.ny + 1) + wr(g, j, g.ny)) * g.nx + wr(g, i, g.nx);
}
__host__ __device__ __forceinline__ int zf(const Geom& g, int k, int j, int i) {
  return g.Fxy + (wr(g, k, g.nz) * g.ny + wr(g, j, g.ny)) * g.nx + wr(g, i, g.nx);
}
__host__ __device__ __forceinline__ int cid(const Geom& g, int k, int j, int i) {
  return (wr(g, k, g.nz) * g.ny + wr(g, j, g.ny)) * g.nx + wr(g, i, g.nx);
}

// interior (non-wall) faces, with the index range check folded in; on a
// periodic grid every neighbour is a face
__device__ __forceinline__ bool xin(const Geom& g, int k, int j, int i) {
  return g.periodic || (i >= 1 && i <= g.nx - 1 && j >= 0 && j < g.ny && k >= 0 && k < g.nz);
}
__device__ __forceinline__ bool yin(const Geom& g, int k, int j, int i) {
  return g.periodic || (j >= 1 && j <= g.ny - 1 && i >= 0 && i < g.nx && k >= 0 && k < g.nz);
}
__device__ __forceinline__ bool zin(const Geom& g, int k, int j, int i) {
  return g.periodic || (k >= 1 && k <= g.nz - 1 && i >= 0 && i < g.nx && j >= 0 && j < g.ny);
}

// decode a face index into (axis, k, j, i)
__device__ __forceinline__ int face_coords(const Geom& g, int f, int& k, int& j, int& i) {
  if (f < g.Fx) {
    const int r = f / (g.nx + 1);
    i = f - r * (g.nx + 1);
    k = r / g.ny;
    j = r - k * g.ny;
    return 0;
  }
  if (f < g.Fxy) {
    const int q = f - g.Fx;
    const int r = q / g.nx;
    i = q - r * g.nx;
    k = r / (g.ny + 1);
    j = r - k * (g.ny + 1);
    return 1;
  }
  const int q = f - g.Fxy;
  const int r = q / g.nx;
  i = q - r * g.nx;
  k = r / g.ny;
  j = r - k * g.ny;
  return 2;
}

template <class T, class R = T>
__device__ __forceinline__ R ldv(const T* v, int f) {
  return R(ld(v + f));
}

// curl components on edges (zero on edges lying in a wall)
template <class T, class R = T>
__device__ __forceinline__ R wx(const Geom& g, const T* v, int k, int j, int i) {
  if (!g.periodic && (j <= 0 || j >= g.ny || k <= 0 || k >= g.nz)) return R(0);
  const R a = ldv<T, R>(v, zf(g, k, j, i)) - ldv<T, R>(v, zf(g, k, j - 1, i));
  const R b = ldv<T, R>(v, yf(g, k, j, i)) - ldv<T, R>(v, yf(g, k - 1, j, i));
  return (a - b) * pick<R>(g.ih, g.ihf);
}
template <class T, class R = T>
__device__ __forceinline__ R wy(const Geom& g, const T* v, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || k <= 0 || k >= g.nz)) return R(0);
  const R a = ldv<T, R>(v, xf(g, k, j, i)) - ldv<T, R>(v, xf(g, k - 1, j, i));
  const R b = ldv<T, R>(v, zf(g, k, j, i)) - ldv<T, R>(v, zf(g, k, j, i - 1));
  return (a - b) * pick<R>(g.ih, g.ihf);
}
template <class T, class R = T>
__device__ __forceinline__ R wz(const Geom& g, const T* v, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || j <= 0 || j >= g.ny)) return R(0);
  const R a = ldv<T, R>(v, yf(g, k, j, i)) - ldv<T, R>(v, yf(g, k, j, i - 1));
  const R b = ldv<T, R>(v, xf(g, k, j, i)) - ldv<T, R>(v, xf(g, k, j - 1, i));
  return (a - b) * pick<R>(g.ih, g.ihf);
}

// The two bilinear terms of Adv at an interior face: O1, V1, O2, V2.
template <class R>
struct Terms {
  R o1, v1, o2, v2;
};

template <class T, class R = T>
__device__ __forceinline__ Terms<R> terms_x(const Geom& g, const T* v, int k, int j, int i) {
  Terms<R> t;
  t.o1 = R(0.5) * (wy<T, R>(g, v, k, j, i) + wy<T, R>(g, v, k + 1, j, i));
  t.v1 = R(0.25) * (ldv<T, R>(v, zf(g, k, j, i - 1)) + ldv<T, R>(v, zf(g, k, j, i)) +
                    ldv<T, R>(v, zf(g, k + 1, j, i - 1)) + ldv<T, R>(v, zf(g, k + 1, j, i)));
  t.o2 = R(0.5) * (wz<T, R>(g, v, k, j, i) + wz<T, R>(g, v, k, j + 1, i));
  t.v2 = R(0.25) * (ldv<T, R>(v, yf(g, k, j, i - 1)) + ldv<T, R>(v, yf(g, k, j, i)) +
                    ldv<T, R>(v, yf(g, k, j + 1, i - 1)) + ldv<T, R>(v, yf(g, k, j + 1, i)));
  return t;
}
template <class T, class R = T>
__device__ __forceinline__ Terms<R> terms_y(const Geom& g, const T* v, int k, int j, int i) {
  Terms<R> t;
  t.o1 = R(0.5) * (wz<T, R>(g, v, k, j, i) + wz<T, R>(g, v, k, j, i + 1));
  t.v1 = R(0.25) * (ldv<T, R>(v, xf(g, k, j - 1, i)) + ldv<T, R>(v, xf(g, k, j - 1, i + 1)) +
                    ldv<T, R>(v, xf(g, k, j, i)) + ldv<T, R>(v, xf(g, k, j, i + 1)));
  t.o2 = R(0.5) * (wx<T, R>(g, v, k, j, i) + wx<T, R>(g, v, k + 1, j, i));
  t.v2 = R(0.25) * (ldv<T, R>(v, zf(g, k, j - 1, i)) + ldv<T, R>(v, zf(g, k, j, i)) +
                    ldv<T, R>(v, zf(g, k + 1, j - 1, i)) + ldv<T, R>(v, zf(g, k + 1, j, i)));
  return t;
}
template <class T, class R = T>
__device__ __forceinline__ Terms<R> terms_z(const Geom& g, const T* v, int k, int j, int i) {
  Terms<R> t;
  t.o1 = R(0.5) * (wx<T, R>(g, v, k, j, i) + wx<T, R>(g, v, k, j + 1, i));
  t.v1 = R(0.25) * (ldv<T, R>(v, yf(g, k - 1, j, i)) + ldv<T, R>(v, yf(g, k - 1, j + 1, i)) +
                    ldv<T, R>(v, yf(g, k, j, i)) + ldv<T, R>(v, yf(g, k, j + 1, i)));
  t.o2 = R(0.5) * (wy<T, R>(g, v, k, j, i) + wy<T, R>(g, v, k, j, i + 1));
  t.v2 = R(0.25) * (ldv<T, R>(v, xf(g, k - 1, j, i)) + ldv<T, R>(v, xf(g, k - 1, j, i + 1)) +
                    ldv<T, R>(v, xf(g, k, j, i)) + ldv<T, R>(v, xf(g, k, j, i + 1)));
  return t;
}

template <class T, class R = T>
__device__ __forceinline__ Terms<R> terms(const Geom& g, const T* v, int axis, int k, int j, int i) {
  return axis == 0 ? terms_x<T, R>(g, v, k, j, i) : (axis == 1 ? terms_y<T, R>(g, v, k, j, i)
                                                               : terms_z<T, R>(g, v, k, j, i));
}

__device__ __forceinline__ bool interior(const Geom& g, int axis, int k, int j, int i) {
  return axis == 0 ? xin(g, k, j, i) : (axis == 1 ? yin(g, k, j, i) : zin(g, k, j, i));
}

// a face unknown at coordinates decoded from a slot (wall faces and, when
// periodic, the unused slot n are not)
__device__ __forceinline__ bool is_face(const Geom& g, int axis, int k, int j, int i) {
  if (g.periodic) return axis == 0 ? i < g.nx : (axis == 1 ? j < g.ny : k < g.nz);
  return interior(g, axis, k, j, i);
}

template <class T>
__device__ __forceinline__ T adv(const Geom& g, const T* v, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const Terms<T> t = terms<T, T>(g, v, axis, k, j, i);
  return t.o1 * t.v1 - t.o2 * t.v2;
}

// ---------------------------------------------------------------------------
// (dAdv/dv)^T u at a face.  With alpha1_f = V1(f) u_f, alpha2_f = -V2(f) u_f
// (the coefficients of the edge means) and beta1_f = O1(f) u_f, beta2_f =
// -O2(f) u_f (the coefficients of the face means) on interior faces f:
//  * the edge part: Q_e = 1/2 sum of the alpha's of the faces whose edge mean
//    holds edge e, then the transposed curl W^T Q;
//  * the face-mean part: 1/4 sum of the beta's of the faces whose face mean
//    holds this face.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T alpha1(const Geom& g, const T* v, const T* u, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  return terms<T, T>(g, v, axis, k, j, i).v1 * ld(u + f);
}
template <class T>
__device__ __forceinline__ T alpha2(const Geom& g, const T* v, const T* u, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  return -terms<T, T>(g, v, axis, k, j, i).v2 * ld(u + f);
}
template <class T>
__device__ __forceinline__ T beta1(const Geom& g, const T* v, const T* u, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  return terms<T, T>(g, v, axis, k, j, i).o1 * ld(u + f);
}
template <class T>
__device__ __forceinline__ T beta2(const Geom& g, const T* v, const T* u, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  return -terms<T, T>(g, v, axis, k, j, i).o2 * ld(u + f);
}

// edge values Q (zero on wall edges, where the curl rows vanish)
// x-edge: omega_x is O2 of y-faces (k,j,i), (k-1,j,i) and O1 of z-faces (k,j,i), (k,j-1,i)
template <class T>
__device__ __forceinline__ T qx(const Geom& g, const T* v, const T* u, int k, int j, int i) {
  if (!g.periodic && (j <= 0 || j >= g.ny || k <= 0 || k >= g.nz)) return T(0);
  return T(0.5) * (alpha2(g, v, u, 1, k, j, i) + alpha2(g, v, u, 1, k - 1, j, i) + alpha1(g, v, u, 2, k, j, i) +
                   alpha1(g, v, u, 2, k, j - 1, i));
}
// y-edge: omega_y is O1 of x-faces (k,j,i), (k-1,j,i) and O2 of z-faces (k,j,i), (k,j,i-1)
template <class T>
__device__ __forceinline__ T qy(const Geom& g, const T* v, const T* u, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || k <= 0 || k >= g.nz)) return T(0);
  return T(0.5) * (alpha1(g, v, u, 0, k, j, i) + alpha1(g, v, u, 0, k - 1, j, i) + alpha2(g, v, u, 2, k, j, i) +
                   alpha2(g, v, u, 2, k, j, i - 1));
}
// z-edge: omega_z is O2 of x-faces (k,j,i), (k,j-1,i) and O1 of y-faces (k,j,i), (k,j,i-1)
template <class T>
__device__ __forceinline__ T qz(const Geom& g, const T* v, const T* u, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || j <= 0 || j >= g.ny)) return T(0);
  return T(0.5) * (alpha2(g, v, u, 0, k, j, i) + alpha2(g, v, u, 0, k, j - 1, i) + alpha1(g, v, u, 1, k, j, i) +
                   alpha1(g, v, u, 1, k, j, i - 1));
}

// (dAdv/dv)^T u at the interior face (axis, k, j, i)
template <class T>
__device__ T jtu(const Geom& g, const T* v, const T* u, int axis, int k, int j, int i) {
  const T ih = pick<T>(g.ih, g.ihf);
  if (axis == 0) {
    // W^T: omega_y(k,j,i) +, omega_y(k+1,j,i) -, omega_z(k,j,i) -, omega_z(k,j+1,i) +
    const T r = (qy(g, v, u, k, j, i) - qy(g, v, u, k + 1, j, i) - qz(g, v, u, k, j, i) + qz(g, v, u, k, j + 1, i)) * ih;
    // face means holding this x-face: V1 of y-faces, V2 of z-faces
    const T s = beta1(g, v, u, 1, k, j, i - 1) + beta1(g, v, u, 1, k, j, i) + beta1(g, v, u, 1, k, j + 1, i - 1) +
                beta1(g, v, u, 1, k, j + 1, i) + beta2(g, v, u, 2, k, j, i - 1) + beta2(g, v, u, 2, k, j, i) +
                beta2(g, v, u, 2, k + 1, j, i - 1) + beta2(g, v, u, 2, k + 1, j, i);
    return r + T(0.25) * s;
  }
  if (axis == 1) {
    // W^T: omega_z(k,j,i) +, omega_z(k,j,i+1) -, omega_x(k,j,i) -, omega_x(k+1,j,i) +
    const T r = (qz(g, v, u, k, j, i) - qz(g, v, u, k, j, i + 1) - qx(g, v, u, k, j, i) + qx(g, v, u, k + 1, j, i)) * ih;
    // V2 of x-faces, V1 of z-faces
    const T s = beta2(g, v, u, 0, k, j, i) + beta2(g, v, u, 0, k, j, i + 1) + beta2(g, v, u, 0, k, j - 1, i) +
                beta2(g, v, u, 0, k, j - 1, i + 1) + beta1(g, v, u, 2, k, j, i) + beta1(g, v, u, 2, k, j - 1, i) +
                beta1(g, v, u, 2, k + 1, j, i) + beta1(g, v, u, 2, k + 1, j - 1, i);
    return r + T(0.25) * s;
  }
  // W^T: omega_x(k,j,i) +, omega_x(k,j+1,i) -, omega_y(k,j,i) -, omega_y(k,j,i+1) +
  const T r = (qx(g, v, u, k, j, i) - qx(g, v, u, k, j + 1, i) - qy(g, v, u, k, j, i) + qy(g, v, u, k, j, i + 1)) * ih;
  // V1 of x-faces, V2 of y-faces
  const T s = beta1(g, v, u, 0, k, j, i) + beta1(g, v, u, 0, k, j, i + 1) + beta1(g, v, u, 0, k - 1, j, i) +
              beta1(g, v, u, 0, k - 1, j, i + 1) + beta2(g, v, u, 1, k, j, i) + beta2(g, v, u, 1, k, j + 1, i) +
              beta2(g, v, u, 1, k - 1, j, i) + beta2(g, v, u, 1, k - 1, j + 1, i);
  return r + T(0.25) * s;
}

// gradient of a centre field at an interior face; divergence at a cell
template <class T>
__device__ __forceinline__ T grad(const Geom& g, const T* p, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int c = cid(g, k, j, i);
  const int cm = axis == 0 ? cid(g, k, j, i - 1) : (axis == 1 ? cid(g, k, j - 1, i) : cid(g, k - 1, j, i));
  return (ld(p + c) - ld(p + cm)) * pick<T>(g.ih, g.ihf);
}

template <class T>
__device__ __forceinline__ T divergence(const Geom& g, const T* v, int k, int j, int i) {
  return (ld(v + xf(g, k, j, i + 1)) - ld(v + xf(g, k, j, i)) + ld(v + yf(g, k, j + 1, i)) - ld(v + yf(g, k, j, i)) +
          ld(v + zf(g, k + 1, j, i)) - ld(v + zf(g, k, j, i))) *
         pick<T>(g.ih, g.ihf);
}

}  // namespace g3
}  // namespace stc
