// NSO residual, SCGS smoother and transfers on the 3D grid (Sec. 4.2-4.3 with
// a third axis).  Same rows, block structure and transfers as the 2D kernels
// of nso_kernels.cu; a cell has 6 faces, so a time block holds 7 unknowns and
// the cells are 8-coloured by the parities of (i, j, k).
#include <mutex>
#include <type_traits>

#include "grid3d.cuh"
#include "stc_kernels.h"

namespace stc {
namespace {

using namespace g3;

// ---------------------------------------------------------------------------
// rows of f (Eq. KKTAO) at an interior face (axis, k, j, i), flat index e
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T row1(const Geom& g, const CState<T>& x, const T* __restrict__ z, int t, int e, int axis,
                                  int k, int j, int i) {
  const T* vt = x.v + (size_t)t * g.F;
  const T* um = x.u + (size_t)(t - 1) * g.F;
  const T* pb = x.pbar + (size_t)t * g.C;
  T val = ld(um + e) * pick<T>(g.idt, g.idtf);
  if (g.self_adv) val += jtu(g, vt, um, axis, k, j, i);
  val += grad(g, pb, axis, k, j, i);
  if (t < g.N) {
    const T* ut = x.u + (size_t)t * g.F;
    val += pick<T>(g.a, g.af) * (ld(vt + e) - ld(z + (size_t)t * g.F + e)) - ld(ut + e) * pick<T>(g.idt, g.idtf);
  }
  return val;
}

template <class T>
__device__ __forceinline__ T row3(const Geom& g, const CState<T>& x, int t, int e, int axis, int k, int j, int i) {
  const T* vn = x.v + (size_t)(t + 1) * g.F;
  const T* vt = x.v + (size_t)t * g.F;
  T val = (ld(vn + e) - ld(vt + e)) * pick<T>(g.idt, g.idtf) - ld(x.u + (size_t)t * g.F + e);
  if (g.self_adv) val += adv(g, vn, axis, k, j, i);
  val += grad(g, x.p + (size_t)t * g.C, axis, k, j, i);
  return val;
}

// ---------------------------------------------------------------------------
// Two-pass form of rows 1 and 3 on large levels.  The Jacobian-transpose term
// (dAdv(v_t)/dv)^T u_{t-1} of row 1 gathers, per face, the products
// alpha1 = V1 u, alpha2 = -V2 u, beta1 = O1 u, beta2 = -O2 u of ~24 faces
// around it, and each product needs the Lamb-vector terms (O1, V1, O2, V2) of
// its own face: evaluated inline per output face, that is ~150 dependent
// loads and thousands of instructions per face, and the kernel was bound by
// instruction fetch.  Pass A (lamb3_terms_kernel, one launch per face axis)
// evaluates the terms of v_t once per face and stores the four products with
// u_{t-1} and Adv(v_t) = O1 V1 - O2 V2; pass B (the residual kernels with
// AB = true) gathers them.  Same sums in the same order as the inline form.
// ---------------------------------------------------------------------------
// the four products of a face in one 16- (fp32) or 32-byte (fp64) record:
// the gathers of row 1 often take two products of the same face (measured:
// records beat four separate planes, 1.25 against 1.33 ms per colour residual)
template <class T>
struct alignas(4 * sizeof(T)) AB4 {
  T a1, a2, b1, b2;
};

// Terms (O1, V1, O2, V2) of an interior face of the closed box from its base
// indices and fixed strides: the same loads, differences and sums in the same
// order as terms_x / terms_y / terms_z of grid3d.cuh, without re-deriving every
// neighbour's index (pass A was bound by that integer arithmetic).  Axes are
// cyclic: for an a-face, b = a+1 and c = a+2; O1 is the mean of the two
// omega_b edges at offsets 0 and +1 along c, V1 the mean of the four c-faces
// at offsets (0, -1 along a) x (0, +1 along c); O2, V2 the same with b, c
// swapped.  lo_c / hi_c: the edge at offset 0 / +1 along c lies in a wall.
__device__ __forceinline__ void box_strides(const Geom& g, int st[3][3]) {
  st[0][0] = 1; st[0][1] = g.nx + 1; st[0][2] = (g.nx + 1) * g.ny;
  st[1][0] = 1; st[1][1] = g.nx;     st[1][2] = g.nx * (g.ny + 1);
  st[2][0] = 1; st[2][1] = g.nx;     st[2][2] = g.nx * g.ny;
}

// omega_b on the edge between faces f_a (axis a) and f_c (axis c) at base
// indices fa, fc, as in wx/wy/wz: (v_a(+0) - v_a(-1 along c)) - (v_c(+0) - v_c(-1 along a)),
// with the sign convention of the component b = a+1
template <class T, int A>
__device__ __forceinline__ T edge_b(const T* v, int fa, int fc, int sa_c, int sc_a, T ih) {
  // A = 0: omega_y = (x(k) - x(k-1)) - (z(i) - z(i-1));  A = 1: omega_z = (y(i) - y(i-1)) - (x(j) - x(j-1));
  // A = 2: omega_x = (z(j) - z(j-1)) - (y(k) - y(k-1))
  const T a = ld(v + fa) - ld(v + fa - sa_c);
  const T b = ld(v + fc) - ld(v + fc - sc_a);
  return (a - b) * ih;
}

// omega_c on the edge between faces f_b and f_a, as in wx/wy/wz:
// (v_b(+0) - v_b(-1 along a)) - (v_a(+0) - v_a(-1 along b))
template <class T>
__device__ __forceinline__ T edge_c(const T* v, int fb, int fa, int sb_a, int sa_b, T ih) {
  const T a = ld(v + fb) - ld(v + fb - sb_a);
  const T b = ld(v + fa) - ld(v + fa - sa_b);
  return (a - b) * ih;
}

// mean of the four faces f + {-sa, 0} x {0, +sp} in the summation order of
// grid3d.cuh: FIRST_A lists both offsets along a at the first +sp offset
// before the second (terms_x), otherwise both +sp offsets at -sa first
template <class T, bool FIRST_A>
__device__ __forceinline__ T mean4(const T* v, int f, int sa, int sp) {
  if (FIRST_A) return T(0.25) * (ld(v + f - sa) + ld(v + f) + ld(v + f + sp - sa) + ld(v + f + sp));
  return T(0.25) * (ld(v + f - sa) + ld(v + f - sa + sp) + ld(v + f) + ld(v + f + sp));
}

template <class T, int A>
__device__ __forceinline__ Terms<T> terms_box(const Geom& g, const T* v, int k, int j, int i) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  int st[3][3];
  box_strides(g, st);
  const int c3[3] = {i, j, k};
  const int n3[3] = {g.nx, g.ny, g.nz};
  const int fa = A == 0 ? xf(g, k, j, i) : (A == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  const int fb = B == 0 ? xf(g, k, j, i) : (B == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  const int fc = C == 0 ? xf(g, k, j, i) : (C == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  const T ih = pick<T>(g.ih, g.ihf);
  Terms<T> t;
  // O1: omega_b edges at offsets 0 and +1 along c (a wall edge when the c coordinate is 0 or n_c)
  const T w0 = c3[C] > 0 ? edge_b<T, A>(v, fa, fc, st[A][C], st[C][A], ih) : T(0);
  const T w1 = c3[C] + 1 < n3[C] ? edge_b<T, A>(v, fa + st[A][C], fc + st[C][C], st[A][C], st[C][A], ih) : T(0);
  t.o1 = T(0.5) * (w0 + w1);
  // V1: c-faces at (a: -1, 0) x (c: 0, +1)
  t.v1 = mean4<T, A == 0>(v, fc, st[C][A], st[C][C]);
  // O2: omega_c edges at offsets 0 and +1 along b
  const T q0 = c3[B] > 0 ? edge_c<T>(v, fb, fa, st[B][A], st[A][B], ih) : T(0);
  const T q1 = c3[B] + 1 < n3[B] ? edge_c<T>(v, fb + st[B][B], fa + st[A][B], st[B][A], st[A][B], ih) : T(0);
  t.o2 = T(0.5) * (q0 + q1);
  // V2: b-faces at (a: -1, 0) x (b: 0, +1)
  t.v2 = mean4<T, A != 2>(v, fb, st[B][A], st[B][B]);
  return t;
}

// pass A: faces of one axis at times t = 0..N (blockIdx.y); AB4 of v_t with
// u_{t-1} for t >= 1, Adv(v_t); zero on slots that are not interior faces
template <class T, int AXIS>
__global__ void __launch_bounds__(128) lamb3_terms_kernel(Geom g, const T* __restrict__ v, const T* __restrict__ u,
                                                          AB4<T>* __restrict__ ab, T* __restrict__ advb) {
  pdl_wait();
  const int t = blockIdx.y;
  const int n0 = AXIS == 0 ? g.nx + 1 : g.nx, n1 = AXIS == 1 ? g.ny + 1 : g.ny;
  const int nf = n0 * n1 * (AXIS == 2 ? g.nz + 1 : g.nz);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nf || t > g.N) return;
  const int i = e % n0, r = e / n0, j = r % n1, k = r / n1;
  const int f = (AXIS == 0 ? 0 : (AXIS == 1 ? g.Fx : g.Fxy)) + e;
  const size_t at = (size_t)t * g.F + f;
  AB4<T> o{T(0), T(0), T(0), T(0)};
  T a = T(0);
  if (interior(g, AXIS, k, j, i)) {
    const Terms<T> tm = g.periodic ? terms<T, T>(g, v + (size_t)t * g.F, AXIS, k, j, i)
                                   : terms_box<T, AXIS>(g, v + (size_t)t * g.F, k, j, i);
    a = tm.o1 * tm.v1 - tm.o2 * tm.v2;
    if (t >= 1) {
      const T uf = ld(u + (size_t)(t - 1) * g.F + f);
      o.a1 = tm.v1 * uf;
      o.a2 = -tm.v2 * uf;
      o.b1 = tm.o1 * uf;
      o.b2 = -tm.o2 * uf;
    }
  }
  ab[at] = o;
  advb[at] = a;
}

// one product of the face (axis, k, j, i) of slice t, zero off the interior faces
// the records of one time slice
template <class T>
using ABt = const AB4<T>*;

template <class T, int C>
__device__ __forceinline__ T abv(const Geom& g, ABt<T> abt, int axis, int k, int j, int i) {
  if (!interior(g, axis, k, j, i)) return T(0);
  const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
  const AB4<T> q = abt[f];
  return C == 0 ? q.a1 : (C == 1 ? q.a2 : (C == 2 ? q.b1 : q.b2));
}

// the edge sums Q from stored products (the same sums as qx, qy, qz)
template <class T>
__device__ __forceinline__ T qx_ab(const Geom& g, ABt<T> a, int k, int j, int i) {
  if (!g.periodic && (j <= 0 || j >= g.ny || k <= 0 || k >= g.nz)) return T(0);
  return T(0.5) * (abv<T, 1>(g, a, 1, k, j, i) + abv<T, 1>(g, a, 1, k - 1, j, i) + abv<T, 0>(g, a, 2, k, j, i) +
                   abv<T, 0>(g, a, 2, k, j - 1, i));
}
template <class T>
__device__ __forceinline__ T qy_ab(const Geom& g, ABt<T> a, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || k <= 0 || k >= g.nz)) return T(0);
  return T(0.5) * (abv<T, 0>(g, a, 0, k, j, i) + abv<T, 0>(g, a, 0, k - 1, j, i) + abv<T, 1>(g, a, 2, k, j, i) +
                   abv<T, 1>(g, a, 2, k, j, i - 1));
}
template <class T>
__device__ __forceinline__ T qz_ab(const Geom& g, ABt<T> a, int k, int j, int i) {
  if (!g.periodic && (i <= 0 || i >= g.nx || j <= 0 || j >= g.ny)) return T(0);
  return T(0.5) * (abv<T, 1>(g, a, 0, k, j, i) + abv<T, 1>(g, a, 0, k, j - 1, i) + abv<T, 0>(g, a, 1, k, j, i) +
                   abv<T, 0>(g, a, 1, k, j, i - 1));
}

// (dAdv/dv)^T u at an interior face from stored products (the order of jtu)
template <class T>
__device__ T jtu_ab(const Geom& g, ABt<T> a, int axis, int k, int j, int i) {
  const T ih = pick<T>(g.ih, g.ihf);
  if (axis == 0) {
    const T r = (qy_ab(g, a, k, j, i) - qy_ab(g, a, k + 1, j, i) - qz_ab(g, a, k, j, i) + qz_ab(g, a, k, j + 1, i)) *
                ih;
    const T s = abv<T, 2>(g, a, 1, k, j, i - 1) + abv<T, 2>(g, a, 1, k, j, i) + abv<T, 2>(g, a, 1, k, j + 1, i - 1) +
                abv<T, 2>(g, a, 1, k, j + 1, i) + abv<T, 3>(g, a, 2, k, j, i - 1) + abv<T, 3>(g, a, 2, k, j, i) +
                abv<T, 3>(g, a, 2, k + 1, j, i - 1) + abv<T, 3>(g, a, 2, k + 1, j, i);
    return r + T(0.25) * s;
  }
  if (axis == 1) {
    const T r = (qz_ab(g, a, k, j, i) - qz_ab(g, a, k, j, i + 1) - qx_ab(g, a, k, j, i) + qx_ab(g, a, k + 1, j, i)) *
                ih;
    const T s = abv<T, 3>(g, a, 0, k, j, i) + abv<T, 3>(g, a, 0, k, j, i + 1) + abv<T, 3>(g, a, 0, k, j - 1, i) +
                abv<T, 3>(g, a, 0, k, j - 1, i + 1) + abv<T, 2>(g, a, 2, k, j, i) + abv<T, 2>(g, a, 2, k, j - 1, i) +
                abv<T, 2>(g, a, 2, k + 1, j, i) + abv<T, 2>(g, a, 2, k + 1, j - 1, i);
    return r + T(0.25) * s;
  }
  const T r = (qx_ab(g, a, k, j, i) - qx_ab(g, a, k, j + 1, i) - qy_ab(g, a, k, j, i) + qy_ab(g, a, k, j, i + 1)) * ih;
  const T s = abv<T, 2>(g, a, 0, k, j, i) + abv<T, 2>(g, a, 0, k, j, i + 1) + abv<T, 2>(g, a, 0, k - 1, j, i) +
              abv<T, 2>(g, a, 0, k - 1, j, i + 1) + abv<T, 3>(g, a, 1, k, j, i) + abv<T, 3>(g, a, 1, k, j + 1, i) +
              abv<T, 3>(g, a, 1, k - 1, j, i) + abv<T, 3>(g, a, 1, k - 1, j + 1, i);
  return r + T(0.25) * s;
}

// The same gather at a face of a closed box at least one cell from the walls
// along every axis (1 <= i, j, k <= n - 2): there every edge sum and every
// product jtu_ab reads is interior, so the wall tests drop out and the records
// sit at fixed offsets from the face's three base indices.  Same sums in the
// same order as jtu_ab.
template <class T>
__device__ __forceinline__ bool jtu_fast_ok(const Geom& g, int k, int j, int i) {
  return !g.periodic && i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2 && k >= 1 && k <= g.nz - 2;
}

template <class T>
__device__ T jtu_ab_far(const Geom& g, ABt<T> a, int axis, int k, int j, int i) {
  const T ih = pick<T>(g.ih, g.ihf);
  const int sxy = g.nx + 1, sxz = (g.nx + 1) * g.ny;   // x-face strides along j, k
  const int syy = g.nx, syz = g.nx * (g.ny + 1);       // y-faces
  const int szy = g.nx, szz = g.nx * g.ny;             // z-faces
  const AB4<T>* X = a + (k * g.ny + j) * sxy + i;
  const AB4<T>* Y = a + g.Fx + (k * (g.ny + 1) + j) * syy + i;
  const AB4<T>* Z = a + g.Fxy + (k * g.ny + j) * szy + i;
  if (axis == 0) {
    const T qy0 = T(0.5) * (X[0].a1 + X[-sxz].a1 + Z[0].a2 + Z[-1].a2);
    const T qy1 = T(0.5) * (X[sxz].a1 + X[0].a1 + Z[szz].a2 + Z[szz - 1].a2);
    const T qz0 = T(0.5) * (X[0].a2 + X[-sxy].a2 + Y[0].a1 + Y[-1].a1);
    const T qz1 = T(0.5) * (X[sxy].a2 + X[0].a2 + Y[syy].a1 + Y[syy - 1].a1);
    const T r = (qy0 - qy1 - qz0 + qz1) * ih;
    const T s = Y[-1].b1 + Y[0].b1 + Y[syy - 1].b1 + Y[syy].b1 + Z[-1].b2 + Z[0].b2 + Z[szz - 1].b2 + Z[szz].b2;
    return r + T(0.25) * s;
  }
  if (axis == 1) {
    const T qz0 = T(0.5) * (X[0].a2 + X[-sxy].a2 + Y[0].a1 + Y[-1].a1);
    const T qz1 = T(0.5) * (X[1].a2 + X[1 - sxy].a2 + Y[1].a1 + Y[0].a1);
    const T qx0 = T(0.5) * (Y[0].a2 + Y[-syz].a2 + Z[0].a1 + Z[-szy].a1);
    const T qx1 = T(0.5) * (Y[syz].a2 + Y[0].a2 + Z[szz].a1 + Z[szz - szy].a1);
    const T r = (qz0 - qz1 - qx0 + qx1) * ih;
    const T s = X[0].b2 + X[1].b2 + X[-sxy].b2 + X[1 - sxy].b2 + Z[0].b1 + Z[-szy].b1 + Z[szz].b1 + Z[szz - szy].b1;
    return r + T(0.25) * s;
  }
  const T qx0 = T(0.5) * (Y[0].a2 + Y[-syz].a2 + Z[0].a1 + Z[-szy].a1);
  const T qx1 = T(0.5) * (Y[syy].a2 + Y[syy - syz].a2 + Z[szy].a1 + Z[0].a1);
  const T qy0 = T(0.5) * (X[0].a1 + X[-sxz].a1 + Z[0].a2 + Z[-1].a2);
  const T qy1 = T(0.5) * (X[1].a1 + X[1 - sxz].a1 + Z[1].a2 + Z[0].a2);
  const T r = (qx0 - qx1 - qy0 + qy1) * ih;
  const T s = X[0].b1 + X[1].b1 + X[-sxz].b1 + X[1 - sxz].b1 + Y[0].b2 + Y[syy].b2 + Y[-syz].b2 + Y[syy - syz].b2;
  return r + T(0.25) * s;
}

// rows 1 and 3 from the stored products (AB) or inline
template <class T, bool AB>
__device__ __forceinline__ T row1x(const Geom& g, const CState<T>& x, const T* __restrict__ z, ABt<T> ab,
                                   int t, int e, int axis, int k, int j, int i) {
  if (!AB) return row1(g, x, z, t, e, axis, k, j, i);
  const T* vt = x.v + (size_t)t * g.F;
  const T* pb = x.pbar + (size_t)t * g.C;
  T val = ld(x.u + (size_t)(t - 1) * g.F + e) * pick<T>(g.idt, g.idtf);
  if (g.self_adv)
    val += jtu_fast_ok<T>(g, k, j, i) ? jtu_ab_far(g, ab + (size_t)t * g.F, axis, k, j, i)
                                      : jtu_ab(g, ab + (size_t)t * g.F, axis, k, j, i);
  val += grad(g, pb, axis, k, j, i);
  if (t < g.N) {
    const T* ut = x.u + (size_t)t * g.F;
    val += pick<T>(g.a, g.af) * (ld(vt + e) - ld(z + (size_t)t * g.F + e)) - ld(ut + e) * pick<T>(g.idt, g.idtf);
  }
  return val;
}

template <class T, bool AB>
__device__ __forceinline__ T row3x(const Geom& g, const CState<T>& x, const T* advb, int t, int e, int axis, int k,
                                   int j, int i) {
  if (!AB) return row3(g, x, t, e, axis, k, j, i);
  const T* vn = x.v + (size_t)(t + 1) * g.F;
  const T* vt = x.v + (size_t)t * g.F;
  T val = (ld(vn + e) - ld(vt + e)) * pick<T>(g.idt, g.idtf) - ld(x.u + (size_t)t * g.F + e);
  if (g.self_adv) val += ld(advb + (size_t)(t + 1) * g.F + e);
  val += grad(g, x.p + (size_t)t * g.C, axis, k, j, i);
  return val;
}

// out = sf * f(x) + sr * res; thread x: face e (< F) and cell e (< C); blockIdx.y: t
template <class T, bool AB>
__global__ void nso_residual3_kernel(Geom g, CState<T> x, const T* __restrict__ z, CState<T> res, State<T> out,
                                     T sf, T sr, double* sq, RedScratch rs, const double* only_if_undone,
                                     const AB4<T>* __restrict__ ab, const T* __restrict__ advb) {
  pdl_wait();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (t > g.N) return;
  if (only_if_undone && only_if_undone[1] <= only_if_undone[0]) return;
  T acc = T(0);
  if (e < g.F) {
    int k, j, i;
    const int axis = face_coords(g, e, k, j, i);
    const bool in = is_face(g, axis, k, j, i);
    if (t >= 1) {
      T val = T(0);
      if (in) {
        val = row1x<T, AB>(g, x, z, ab, t, e, axis, k, j, i) * sf;
        if (res.v) val += sr * ld(res.v + (size_t)t * g.F + e);
      }
      out.v[(size_t)t * g.F + e] = val;
      acc += val * val;
    } else {
      out.v[e] = T(0);
    }
    if (t < g.N) {
      T val = T(0);
      if (in) {
        val = row3x<T, AB>(g, x, advb, t, e, axis, k, j, i) * sf;
        if (res.u) val += sr * ld(res.u + (size_t)t * g.F + e);
      }
      out.u[(size_t)t * g.F + e] = val;
      acc += val * val;
    }
  }
  if (e < g.C) {
    const int i = e % g.nx, r = e / g.nx, j = r % g.ny, k = r / g.ny;
    if (t >= 1) {
      T val = -divergence(g, x.v + (size_t)t * g.F, k, j, i) * sf;
      if (res.pbar) val += sr * ld(res.pbar + (size_t)t * g.C + e);
      out.pbar[(size_t)t * g.C + e] = val;
      acc += val * val;
    } else {
      out.pbar[e] = T(0);
    }
    if (t < g.N) {
      T val = -divergence(g, x.u + (size_t)t * g.F, k, j, i) * sf;
      if (res.p) val += sr * ld(res.p + (size_t)t * g.C + e);
      out.p[(size_t)t * g.C + e] = val;
      acc += val * val;
    }
  }
  if (sq) block_sum_ordered((double)acc, sq, rs);
}

// f - res at what one colour's SCGS reads: the faces of its cells (x-faces of
// rows j = py, k = pz (mod 2); y-faces of i = px, k = pz; z-faces of i = px,
// j = py) and its cells.  Thread x: index over those; blockIdx.y: t.
template <class T, bool AB>
__global__ void nso_residual3_colour_kernel(Geom g, CState<T> x, const T* __restrict__ z, CState<T> res,
                                            State<T> out, int px, int py, int pz, const double* only_if_undone,
                                            const AB4<T>* __restrict__ ab, const T* __restrict__ advb) {
  pdl_wait();
  const int t = blockIdx.y;
  if (t > g.N) return;
  if (only_if_undone && only_if_undone[1] <= only_if_undone[0]) return;
  const int ncx = (g.nx - px + 1) / 2, ncy = (g.ny - py + 1) / 2, ncz = (g.nz - pz + 1) / 2;
  const int nxf = ncz * ncy * (g.nx + 1), nyf = ncz * (g.ny + 1) * ncx, nzf = (g.nz + 1) * ncy * ncx;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nxf + nyf + nzf) {
    int axis, k, j, i;
    if (e < nxf) {
      axis = 0;
      i = e % (g.nx + 1);
      const int r = e / (g.nx + 1);
      j = py + 2 * (r % ncy);
      k = pz + 2 * (r / ncy);
    } else if (e < nxf + nyf) {
      axis = 1;
      const int q = e - nxf;
      i = px + 2 * (q % ncx);
      const int r = q / ncx;
      j = r % (g.ny + 1);
      k = pz + 2 * (r / (g.ny + 1));
    } else {
      axis = 2;
      const int q = e - nxf - nyf;
      i = px + 2 * (q % ncx);
      const int r = q / ncx;
      j = py + 2 * (r % ncy);
      k = r / ncy;
    }
    // (the unused slot n of a periodic axis aliases face 0: its rows stay untouched)
    if (g.periodic && !is_face(g, axis, k, j, i)) return;
    const int f = axis == 0 ? xf(g, k, j, i) : (axis == 1 ? yf(g, k, j, i) : zf(g, k, j, i));
    const bool in = is_face(g, axis, k, j, i);
    if (t >= 1) {
      T val = T(0);
      if (in) {
        val = row1x<T, AB>(g, x, z, ab, t, f, axis, k, j, i);
        if (res.v) val -= ld(res.v + (size_t)t * g.F + f);
      }
      out.v[(size_t)t * g.F + f] = val;
    }
    if (t < g.N) {
      T val = T(0);
      if (in) {
        val = row3x<T, AB>(g, x, advb, t, f, axis, k, j, i);
        if (res.u) val -= ld(res.u + (size_t)t * g.F + f);
      }
      out.u[(size_t)t * g.F + f] = val;
    }
    return;
  }
  e -= nxf + nyf + nzf;
  if (e < ncx * ncy * ncz) {
    const int i = px + 2 * (e % ncx), r = e / ncx, j = py + 2 * (r % ncy), k = pz + 2 * (r / ncy);
    const int c = cid(g, k, j, i);
    if (t >= 1) {
      T val = -divergence(g, x.v + (size_t)t * g.F, k, j, i);
      if (res.pbar) val -= ld(res.pbar + (size_t)t * g.C + c);
      out.pbar[(size_t)t * g.C + c] = val;
    }
    if (t < g.N) {
      T val = -divergence(g, x.u + (size_t)t * g.F, k, j, i);
      if (res.p) val -= ld(res.p + (size_t)t * g.C + c);
      out.p[(size_t)t * g.C + c] = val;
    }
  }
}

// ---------------------------------------------------------------------------
// SCGS on the 3D grid.  Local faces a = 0..5: (x-, x+, y-, y+, z-, z+) of the
// cell, axis a / 2, side a % 2.  Block structure and phases as in the 2D
// kernel (nso_kernels.cu): all u blocks eliminated in closed form, cyclic
// reduction over the N v blocks (one warp per cell), u blocks recovered.
// ---------------------------------------------------------------------------
constexpr int NF = 6;                 // faces per cell
constexpr int NB = NF + 1;            // unknowns per time block
constexpr int NSYM = NF * (NF + 1) / 2;
constexpr int NRHS = 2 * NF + 1;      // saddle solves in the reduction: two couplings + rhs
enum : int {
  C3_A = 0,                       // symmetric face block (NSYM)
  C3_R = C3_A + NSYM,             // right-hand side (NB)
  C3_C = C3_R + NB,               // coupling to the next block (NF x NF)
  C3_ZL = C3_C + NF * NF,         // solved left coupling (NF x NF) + its multipliers (NF)
  C3_ZR = C3_ZL + NF * NF + NF,   // solved right coupling + multipliers
  C3_Z = C3_ZR + NF * NF + NF,    // solved right-hand side (NB)
  kCr3Stride = C3_Z + NB          // 155: odd, so a warp's lanes hit distinct banks
};
static_assert(kCr3Stride % 2 == 1, "record stride must be odd");

__host__ __device__ inline size_t scgs3_cell_floats(int N) { return (size_t)(NF * NF + NB + kCr3Stride) * N; }

template <class S>
struct CellG3 {
  S act[NF], g[NF], gh[NF], ig2;
  __device__ void init(const Geom& geo, int i, int j, int k) {
    const bool pr = geo.periodic != 0;   // no walls: every face of every cell is an unknown
    act[0] = S(pr || i > 0);
    act[1] = S(pr || i < geo.nx - 1);
    act[2] = S(pr || j > 0);
    act[3] = S(pr || j < geo.ny - 1);
    act[4] = S(pr || k > 0);
    act[5] = S(pr || k < geo.nz - 1);
    S g2 = S(0);
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      g[a] = ((a & 1) ? -act[a] : act[a]) * S(geo.ih);
      g2 += g[a] * g[a];
    }
    ig2 = S(1) / g2;
#pragma unroll
    for (int a = 0; a < NF; ++a) gh[a] = g[a] * ig2;
  }
  __device__ __forceinline__ void proj(const S w[NF], S out[NF]) const {
    S d = S(0);
#pragma unroll
    for (int a = 0; a < NF; ++a) d += g[a] * w[a];
#pragma unroll
    for (int a = 0; a < NF; ++a) out[a] = act[a] * w[a] - gh[a] * d;
  }
};

// d Adv_f / d v_g for f, g among the 6 faces of cell (k, j, i) at field v.
// Face f = (A, s) carries two terms: +O1 V1 with omega component C = A+1 and
// face mean of component B = A+2, and -O2 V2 with C = A+2, B = A+1 (cyclic).
// The C-edges on f lie at its two ends along B, at the corners with the
// cell's faces (B, d); such an edge is interior iff neither face plane is a
// wall.  Its curl stencil holds two of the cell's faces: (A, s) with weight
// c(C, A, d) and (B, d) with weight c(C, B, s), where
//   c(C, X, side) = (X == C+2 ? +1 : -1) * (side == 0 ? +1 : -1) / h.
// The face mean of component B holds the cell's two B-faces with weight 1/4.
template <class T, class R>
__device__ void local_adv_jac3(const Geom& g, const T* v, int k, int j, int i, const R act[NF], R J[NF][NF]) {
  const R ih = pick<R>(g.ih, g.ihf);
#pragma unroll
  for (int r = 0; r < NF; ++r)
#pragma unroll
    for (int c = 0; c < NF; ++c) J[r][c] = R(0);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int A = f >> 1, s = f & 1;
    const int fk = k + (A == 2 ? s : 0), fj = j + (A == 1 ? s : 0), fi = i + (A == 0 ? s : 0);
    if (!interior(g, A, fk, fj, fi)) continue;
    Terms<R> tm;
    if constexpr (std::is_same<T, R>::value) {   // closed box: the strength-reduced form of pass A
      if (!g.periodic)
        tm = A == 0 ? terms_box<T, 0>(g, v, fk, fj, fi)
                    : (A == 1 ? terms_box<T, 1>(g, v, fk, fj, fi) : terms_box<T, 2>(g, v, fk, fj, fi));
      else
        tm = terms<T, R>(g, v, A, fk, fj, fi);
    } else {
      tm = terms<T, R>(g, v, A, fk, fj, fi);
    }
#pragma unroll
    for (int term = 0; term < 2; ++term) {
      const int C = term == 0 ? (A + 1) % 3 : (A + 2) % 3;
      const int B = term == 0 ? (A + 2) % 3 : (A + 1) % 3;
      const R sgn = term == 0 ? R(1) : R(-1);
      const R O = term == 0 ? tm.o1 : tm.o2;
      const R V = term == 0 ? tm.v1 : tm.v2;
      const R sA = (A == (C + 2) % 3) ? R(1) : R(-1);
      const R sB = (B == (C + 2) % 3) ? R(1) : R(-1);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const R ae = act[f] * act[2 * B + d];
        const R dside = d == 0 ? R(1) : R(-1);
        const R sside = s == 0 ? R(1) : R(-1);
        // d O / d v_(A,s) and d O / d v_(B,d)
        J[f][f] += sgn * V * R(0.5) * ae * sA * dside * ih;
        J[f][2 * B + d] += sgn * (V * R(0.5) * ae * sB * sside * ih + O * R(0.25));
      }
    }
  }
}

// Solve [[A, g], [g^T, 0]] [X; y] = [B; q] for NC right-hand sides (A the
// symmetric definite NF x NF face block): LDL^T, the NC columns and g, then
// the Schur step on g.  On return B holds X and Y holds y.
template <class S, int NC>
__device__ __forceinline__ void saddle_solve6(S A[NF][NF], const S gv[NF], S B[NF][NC], const S q[NC], S Y[NC]) {
  S dinv[NF];
#pragma unroll
  for (int kk = 0; kk < NF; ++kk) {
    S d = A[kk][kk];
#pragma unroll
    for (int s = 0; s < kk; ++s) d -= A[kk][s] * A[kk][s] * A[s][s];
    A[kk][kk] = d;
    const S id = S(1) / d;
    dinv[kk] = id;
#pragma unroll
    for (int r = kk + 1; r < NF; ++r) {
      S l = A[r][kk];
#pragma unroll
      for (int s = 0; s < kk; ++s) l -= A[r][s] * A[kk][s] * A[s][s];
      A[r][kk] = l * id;
    }
  }
  S X[NF][NC + 1];
#pragma unroll
  for (int r = 0; r < NF; ++r) {
#pragma unroll
    for (int c = 0; c < NC; ++c) X[r][c] = B[r][c];
    X[r][NC] = gv[r];
  }
#pragma unroll
  for (int c = 0; c <= NC; ++c) {
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      S s = X[r][c];
#pragma unroll
      for (int kk = 0; kk < r; ++kk) s -= A[r][kk] * X[kk][c];
      X[r][c] = s;
    }
#pragma unroll
    for (int r = 0; r < NF; ++r) X[r][c] *= dinv[r];
#pragma unroll
    for (int r = NF - 1; r >= 0; --r) {
      S s = X[r][c];
#pragma unroll
      for (int kk = r + 1; kk < NF; ++kk) s -= A[kk][r] * X[kk][c];
      X[r][c] = s;
    }
  }
  S sgg = S(0);
#pragma unroll
  for (int r = 0; r < NF; ++r) sgg += gv[r] * X[r][NC];
  const S isgg = S(1) / sgg;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    S sgb = S(0);
#pragma unroll
    for (int r = 0; r < NF; ++r) sgb += gv[r] * X[r][c];
    const S y = (sgb - q[c]) * isgg;
    Y[c] = y;
#pragma unroll
    for (int r = 0; r < NF; ++r) B[r][c] = X[r][c] - X[r][NC] * y;
  }
}

template <class S>
__device__ __forceinline__ void load_sym6(const S* v, S A[NF][NF]) {
  int e = 0;
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int b = a; b < NF; ++b) {
      A[a][b] = v[e];
      A[b][a] = v[e];
      ++e;
    }
}

template <class S>
__device__ __forceinline__ void store_sym6(S* v, const S A[NF][NF]) {
  int e = 0;
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int b = a; b < NF; ++b) {
      v[e] = S(0.5) * (A[a][b] + A[b][a]);
      ++e;
    }
}

// shift A by gamma g g^T (gamma from the trace; x unchanged, the multiplier
// shifted by gamma q) and symmetrise; returns gamma
template <class S>
__device__ __forceinline__ S shift_sym6(S A[NF][NF], const CellG3<S>& cg) {
  S tr = S(0);
#pragma unroll
  for (int a = 0; a < NF; ++a) tr += A[a][a];
  const S gam = tr * cg.ig2 / S(NF);
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int b = a; b < NF; ++b) {
      const S m = S(0.5) * (A[a][b] + A[b][a]) + gam * cg.g[a] * cg.g[b];
      A[a][b] = m;
      A[b][a] = m;
    }
  return gam;
}

struct Cell3 {
  int i, j, k;
};

__device__ __forceinline__ Cell3 colour_cell(const Geom& g, int colour, int q) {
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int ncx = (g.nx - px + 1) / 2, ncy = (g.ny - py + 1) / 2;
  Cell3 c;
  c.i = px + 2 * (q % ncx);
  const int r = q / ncx;
  c.j = py + 2 * (r % ncy);
  c.k = pz + 2 * (r / ncy);
  return c;
}

template <class T, class S>
__global__ void __launch_bounds__(256)
scgs3_colour_kernel(Geom g, State<T> x, CState<T> r, int colour, int ncell, int cpb, const double* __restrict__ lm_dev,
                    const S* __restrict__ ubuf) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.N;
  const S lm = S(lm_dev ? *lm_dev : g.lm);
  const int q0 = blockIdx.x * cpb;
  S* Us = reinterpret_cast<S*>(smem_raw);            // U_t        [N][36][cpb]
  S* Bu = Us + (size_t)N * NF * NF * cpb;            // b_u -> y_t [N][7][cpb]
  S* Vb = Bu + (size_t)N * NB * cpb;                 // v blocks   [cpb][N][kCr3Stride]
  const S idt = pick<S>(g.idt, g.idtf);

  // ---- phase A: couplings and right-hand sides ----------------------------
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const Cell3 cl = colour_cell(g, colour, q);
    const int fidx[NF] = {xf(g, cl.k, cl.j, cl.i), xf(g, cl.k, cl.j, cl.i + 1), yf(g, cl.k, cl.j, cl.i),
                          yf(g, cl.k, cl.j + 1, cl.i), zf(g, cl.k, cl.j, cl.i), zf(g, cl.k + 1, cl.j, cl.i)};
    const bool pr = g.periodic != 0;
    S act[NF] = {S(pr || cl.i > 0), S(pr || cl.i < g.nx - 1), S(pr || cl.j > 0), S(pr || cl.j < g.ny - 1),
                 S(pr || cl.k > 0), S(pr || cl.k < g.nz - 1)};
    const int cc = cid(g, cl.k, cl.j, cl.i);
    S* U = Us + (size_t)t * NF * NF * cpb + c;
    if (ubuf) {   // the couplings precomputed for the colour ([t][36][ncell], scgs3t_coupling_kernel)
#pragma unroll
      for (int e = 0; e < NF * NF; ++e) U[e * cpb] = ubuf[((size_t)t * NF * NF + e) * ncell + q];
    } else {
      S Jl[NF][NF];
      local_adv_jac3<T, S>(g, x.v + (size_t)(t + 1) * g.F, cl.k, cl.j, cl.i, act, Jl);
#pragma unroll
      for (int a2 = 0; a2 < NF; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < NF; ++b2)
          U[(a2 * NF + b2) * cpb] = ((a2 == b2 ? idt : S(0)) + S(g.self_adv) * Jl[a2][b2]) * act[a2] * act[b2];
    }
    S* Ru = Bu + (size_t)t * NB * cpb + c;
    S* Rv = Vb + ((size_t)c * N + t) * kCr3Stride + C3_R;
    const T* ru = r.u + (size_t)t * g.F;
    const T* rv = r.v + (size_t)(t + 1) * g.F;
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) {
      Ru[a2 * cpb] = S(-ld(ru + fidx[a2])) * act[a2];
      Rv[a2] = S(-ld(rv + fidx[a2])) * act[a2];
    }
    Ru[NF * cpb] = S(-ld(r.p + (size_t)t * g.C + cc));
    Rv[NF] = S(-ld(r.pbar + (size_t)(t + 1) * g.C + cc));
  }
  __syncthreads();

  // ---- phase A2: eliminate the u blocks ------------------------------------
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const Cell3 cl = colour_cell(g, colour, q);
    CellG3<S> cg_;
    cg_.init(g, cl.i, cl.j, cl.k);
    S* Ru = Bu + (size_t)t * NB * cpb + c;
    S bf[NF], pb[NF];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) bf[a2] = Ru[a2 * cpb];
    const S bp = Ru[NF * cpb];
    cg_.proj(bf, pb);
    S gb = S(0);
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) gb += cg_.gh[a2] * bf[a2];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) Ru[a2 * cpb] = -pb[a2] + cg_.gh[a2] * bp;
    Ru[NF * cpb] = gb + bp * cg_.ig2;
  }
  __syncthreads();
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const Cell3 cl = colour_cell(g, colour, q);
    CellG3<S> cg_;
    cg_.init(g, cl.i, cl.j, cl.k);
    const int tv = t + 1;
    S* V = Vb + ((size_t)c * N + t) * kCr3Stride;
    const S* U = Us + (size_t)t * NF * NF * cpb + c;
    S Um[NF][NF];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < NF; ++b2) Um[a2][b2] = U[(a2 * NF + b2) * cpb];
    S PU[NF][NF];
#pragma unroll
    for (int b2 = 0; b2 < NF; ++b2) {
      S w[NF], pw[NF];
#pragma unroll
      for (int a2 = 0; a2 < NF; ++a2) w[a2] = Um[a2][b2];
      cg_.proj(w, pw);
#pragma unroll
      for (int a2 = 0; a2 < NF; ++a2) PU[a2][b2] = pw[a2];
    }
    const S diag = (tv < N ? pick<S>(g.a, g.af) : S(0)) + lm;
    int e = 0;
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2)
#pragma unroll
      for (int b2 = a2; b2 < NF; ++b2) {
        S v = S(0);
#pragma unroll
        for (int c2 = 0; c2 < NF; ++c2) v += Um[c2][a2] * PU[c2][b2];
        if (tv < N) v += ((a2 == b2 ? cg_.act[a2] : S(0)) - cg_.gh[a2] * cg_.g[b2]) * idt * idt;
        if (a2 == b2) v += cg_.act[a2] > S(0) ? diag : S(1);
        V[C3_A + e] = v;
        ++e;
      }
    const S* y0 = Bu + (size_t)t * NB * cpb + c;
    S yv[NF];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) yv[a2] = y0[a2 * cpb];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) {
      S v = V[C3_R + a2];
#pragma unroll
      for (int c2 = 0; c2 < NF; ++c2) v -= Um[c2][a2] * yv[c2];
      if (tv < N) v += idt * cg_.act[a2] * Bu[((size_t)tv * NB + a2) * cpb + c];
      V[C3_R + a2] = v;
    }
    if (tv < N) {
      const S* U1 = Us + (size_t)tv * NF * NF * cpb + c;
#pragma unroll
      for (int b2 = 0; b2 < NF; ++b2) {
        S w[NF], pw[NF];
#pragma unroll
        for (int a2 = 0; a2 < NF; ++a2) w[a2] = U1[(a2 * NF + b2) * cpb];
        cg_.proj(w, pw);
#pragma unroll
        for (int a2 = 0; a2 < NF; ++a2) V[C3_C + a2 * NF + b2] = -idt * pw[a2];
      }
    } else {
#pragma unroll
      for (int e2 = 0; e2 < NF * NF; ++e2) V[C3_C + e2] = S(0);
    }
  }
  __syncthreads();

  // ---- phase B: cyclic reduction over the v blocks, one warp per cell -------
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = q0 + warp;
    if (warp < cpb && q < ncell) {
      const Cell3 cl = colour_cell(g, colour, q);
      CellG3<S> cg_;
      cg_.init(g, cl.i, cl.j, cl.k);
      S* V = Vb + (size_t)warp * N * kCr3Stride;
      int top = 0;
      for (int s2 = 1; s2 < N; s2 <<= 1) {
        top = s2;
        for (int m = lane;; m += 32) {
          const int o = s2 * (2 * m + 1);
          if (o >= N) break;
          const bool hasb = o + s2 < N;
          S* Vo = V + (size_t)o * kCr3Stride;
          const S* Va = V + (size_t)(o - s2) * kCr3Stride;
          S A[NF][NF];
          load_sym6(Vo + C3_A, A);
          S B[NF][NRHS];
          S qv[NRHS];
#pragma unroll
          for (int r2 = 0; r2 < NF; ++r2) {
#pragma unroll
            for (int c2 = 0; c2 < NF; ++c2) {
              B[r2][c2] = Va[C3_C + c2 * NF + r2];
              B[r2][NF + c2] = hasb ? Vo[C3_C + r2 * NF + c2] : S(0);
            }
            B[r2][2 * NF] = Vo[C3_R + r2];
          }
#pragma unroll
          for (int c2 = 0; c2 < 2 * NF; ++c2) qv[c2] = S(0);
          qv[2 * NF] = Vo[C3_R + NF];
          const S gam = shift_sym6(A, cg_);
          S Y[NRHS];
          saddle_solve6<S, NRHS>(A, cg_.g, B, qv, Y);
          Y[2 * NF] += gam * qv[2 * NF];
#pragma unroll
          for (int c2 = 0; c2 < NF; ++c2) {
#pragma unroll
            for (int r2 = 0; r2 < NF; ++r2) {
              Vo[C3_ZL + r2 * NF + c2] = B[r2][c2];
              Vo[C3_ZR + r2 * NF + c2] = B[r2][NF + c2];
            }
            Vo[C3_ZL + NF * NF + c2] = Y[c2];
            Vo[C3_ZR + NF * NF + c2] = Y[NF + c2];
          }
#pragma unroll
          for (int r2 = 0; r2 < NF; ++r2) Vo[C3_Z + r2] = B[r2][2 * NF];
          Vo[C3_Z + NF] = Y[2 * NF];
        }
        __syncwarp();
        for (int m = lane;; m += 32) {
          const int e = 2 * s2 * m;
          if (e >= N) break;
          S* Ve = V + (size_t)e * kCr3Stride;
          S A[NF][NF];
          load_sym6(Ve + C3_A, A);
          S rf[NF], Ce[NF][NF], Cn[NF][NF];
#pragma unroll
          for (int r2 = 0; r2 < NF; ++r2) {
            rf[r2] = Ve[C3_R + r2];
#pragma unroll
            for (int c2 = 0; c2 < NF; ++c2) {
              Ce[r2][c2] = Ve[C3_C + r2 * NF + c2];
              Cn[r2][c2] = S(0);
            }
          }
          const int o2 = e + s2;
          if (o2 < N) {
            const S* V2 = V + (size_t)o2 * kCr3Stride;
            const bool hasb2 = o2 + s2 < N;
#pragma unroll
            for (int r2 = 0; r2 < NF; ++r2) {
#pragma unroll
              for (int c2 = 0; c2 < NF; ++c2) {
                S aL = S(0), aR = S(0);
#pragma unroll
                for (int k2 = 0; k2 < NF; ++k2) {
                  aL += Ce[r2][k2] * V2[C3_ZL + k2 * NF + c2];
                  aR += Ce[r2][k2] * V2[C3_ZR + k2 * NF + c2];
                }
                A[r2][c2] -= aL;
                Cn[r2][c2] = hasb2 ? -aR : S(0);
              }
              S az = S(0);
#pragma unroll
              for (int k2 = 0; k2 < NF; ++k2) az += Ce[r2][k2] * V2[C3_Z + k2];
              rf[r2] -= az;
            }
          }
          const int o1 = e - s2;
          if (o1 >= 0) {
            const S* V1 = V + (size_t)o1 * kCr3Stride;
#pragma unroll
            for (int r2 = 0; r2 < NF; ++r2) {
#pragma unroll
              for (int c2 = 0; c2 < NF; ++c2) {
                S aR = S(0);
#pragma unroll
                for (int k2 = 0; k2 < NF; ++k2) aR += V1[C3_C + k2 * NF + r2] * V1[C3_ZR + k2 * NF + c2];
                A[r2][c2] -= aR;
              }
              S az = S(0);
#pragma unroll
              for (int k2 = 0; k2 < NF; ++k2) az += V1[C3_C + k2 * NF + r2] * V1[C3_Z + k2];
              rf[r2] -= az;
            }
          }
          store_sym6(Ve + C3_A, A);
#pragma unroll
          for (int r2 = 0; r2 < NF; ++r2) {
            Ve[C3_R + r2] = rf[r2];
#pragma unroll
            for (int c2 = 0; c2 < NF; ++c2) Ve[C3_C + r2 * NF + c2] = Cn[r2][c2];
          }
        }
        __syncwarp();
      }
      if (lane == 0) {
        S A[NF][NF];
        load_sym6(V + C3_A, A);
        S B[NF][1];
        S qv[1] = {V[C3_R + NF]};
#pragma unroll
        for (int r2 = 0; r2 < NF; ++r2) B[r2][0] = V[C3_R + r2];
        const S gam = shift_sym6(A, cg_);
        S Y[1];
        saddle_solve6<S, 1>(A, cg_.g, B, qv, Y);
#pragma unroll
        for (int r2 = 0; r2 < NF; ++r2) V[C3_Z + r2] = B[r2][0];
        V[C3_Z + NF] = Y[0] + gam * qv[0];
      }
      __syncwarp();
      for (int s2 = top; s2 >= 1; s2 >>= 1) {
        for (int m = lane;; m += 32) {
          const int o = s2 * (2 * m + 1);
          if (o >= N) break;
          S* Vo = V + (size_t)o * kCr3Stride;
          const S* Va = V + (size_t)(o - s2) * kCr3Stride;
          const bool hasb = o + s2 < N;
          S xa[NF], xb[NF];
#pragma unroll
          for (int k2 = 0; k2 < NF; ++k2) {
            xa[k2] = Va[C3_Z + k2];
            xb[k2] = hasb ? V[(size_t)(o + s2) * kCr3Stride + C3_Z + k2] : S(0);
          }
#pragma unroll
          for (int r2 = 0; r2 < NB; ++r2) {
            S v = Vo[C3_Z + r2];
#pragma unroll
            for (int k2 = 0; k2 < NF; ++k2) v -= Vo[C3_ZL + r2 * NF + k2] * xa[k2] + Vo[C3_ZR + r2 * NF + k2] * xb[k2];
            Vo[C3_Z + r2] = v;
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // ---- phase C: u blocks from the v solution, x += omega * delta -----------
  const T om = pick<T>(g.omega, g.omegaf);
  for (int item = threadIdx.x; item < cpb * N; item += blockDim.x) {
    const int c = item % cpb, t = item / cpb;
    const int q = q0 + c;
    if (q >= ncell) continue;
    const Cell3 cl = colour_cell(g, colour, q);
    const int fidx[NF] = {xf(g, cl.k, cl.j, cl.i), xf(g, cl.k, cl.j, cl.i + 1), yf(g, cl.k, cl.j, cl.i),
                          yf(g, cl.k, cl.j + 1, cl.i), zf(g, cl.k, cl.j, cl.i), zf(g, cl.k + 1, cl.j, cl.i)};
    const bool pr = g.periodic != 0;
    const bool actb[NF] = {pr || cl.i > 0, pr || cl.i < g.nx - 1, pr || cl.j > 0, pr || cl.j < g.ny - 1,
                           pr || cl.k > 0, pr || cl.k < g.nz - 1};
    const int cc = cid(g, cl.k, cl.j, cl.i);
    T* fu = x.u + (size_t)t * g.F;
    T* fv = x.v + (size_t)(t + 1) * g.F;
    T* fp = x.p + (size_t)t * g.C + cc;
    T* fpb = x.pbar + (size_t)(t + 1) * g.C + cc;
    T old_u[NF], old_v[NF];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) {
      old_u[a2] = actb[a2] ? fu[fidx[a2]] : T(0);
      old_v[a2] = actb[a2] ? fv[fidx[a2]] : T(0);
    }
    const T old_p = *fp, old_pb = *fpb;
    CellG3<S> cg_;
    cg_.init(g, cl.i, cl.j, cl.k);
    const S* U = Us + (size_t)t * NF * NF * cpb + c;
    const S* xv1 = Vb + ((size_t)c * N + t) * kCr3Stride + C3_Z;
    const S* xv0 = Vb + ((size_t)c * N + (t > 0 ? t - 1 : 0)) * kCr3Stride + C3_Z;
    S w[NF];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) {
      S v = S(0);
#pragma unroll
      for (int b2 = 0; b2 < NF; ++b2) v -= U[(a2 * NF + b2) * cpb] * xv1[b2];
      if (t >= 1) v += idt * cg_.act[a2] * xv0[a2];
      w[a2] = v;
    }
    S pw[NF];
    cg_.proj(w, pw);
    S gw = S(0);
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) gw += cg_.gh[a2] * w[a2];
    const S* y = Bu + (size_t)t * NB * cpb + c;
    S du[NB];
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2) du[a2] = y[a2 * cpb] - pw[a2];
    du[NF] = y[NF * cpb] + gw;
#pragma unroll
    for (int a2 = 0; a2 < NF; ++a2)
      if (actb[a2]) {
        fu[fidx[a2]] = old_u[a2] + om * T(du[a2]);
        fv[fidx[a2]] = old_v[a2] + om * T(xv1[a2]);
      }
    *fp = old_p + om * T(du[NF]);
    *fpb = old_pb + om * T(xv1[NF]);
  }
}

// ---------------------------------------------------------------------------
// SCGS on the 3D grid, one thread per cell: the same local system (u blocks
// eliminated in closed form, N symmetric saddle v blocks coupled by
// O_t = -P U_{t+1} / dt) solved by block Thomas elimination along time, the
// O(N) solve of Sec. 4.3.  A level with many cells per colour has parallelism
// enough across cells, and this form does about half the arithmetic of the
// cyclic reduction with no shared memory.  Each thread streams its pivots'
// solutions (Z_t = A_t^{-1} [O_t; 0] and z_t = A_t^{-1} r_t, 49 values per
// block) to a scratch laid out cell-fastest, so the accesses of a warp are
// coalesced.  Passes: (1) ascending elimination, (2) descending
// substitution x_t = z_t - Z_t x_{t+1} in place, (3) ascending recovery of
// the u blocks and x += omega delta.  The couplings U_t come precomputed
// (scgs3t_coupling_kernel) and every global value a step reads is copied
// into shared memory one step ahead, so the recurrence waits on no load.
// ---------------------------------------------------------------------------
constexpr int kThomasRec = NF * NF + NF + NB;   // X (6x6), multipliers (6), z (7)
constexpr int kThomasCpl = NF * NF;             // U_t of one cell and step (6x6)

template <class T, class S>
struct ThomasCell {
  const Geom& g;
  int fidx[NF], cc;
  S act[NF];
  Cell3 cl;
  __device__ ThomasCell(const Geom& g_, int colour, int q) : g(g_) {
    cl = colour_cell(g, colour, q);
    fidx[0] = xf(g, cl.k, cl.j, cl.i);
    fidx[1] = xf(g, cl.k, cl.j, cl.i + 1);
    fidx[2] = yf(g, cl.k, cl.j, cl.i);
    fidx[3] = yf(g, cl.k, cl.j + 1, cl.i);
    fidx[4] = zf(g, cl.k, cl.j, cl.i);
    fidx[5] = zf(g, cl.k + 1, cl.j, cl.i);
    const bool pr = g.periodic != 0;
    act[0] = S(pr || cl.i > 0);
    act[1] = S(pr || cl.i < g.nx - 1);
    act[2] = S(pr || cl.j > 0);
    act[3] = S(pr || cl.j < g.ny - 1);
    act[4] = S(pr || cl.k > 0);
    act[5] = S(pr || cl.k < g.nz - 1);
    cc = cid(g, cl.k, cl.j, cl.i);
  }
  // U_t = (I/dt + dAdv_loc(v_{t+1})) on the active face pairs
  __device__ void coupling(const T* v_t1, S idt, S U[NF][NF]) const {
    local_adv_jac3<T, S>(g, v_t1, cl.k, cl.j, cl.i, act, U);
#pragma unroll
    for (int a = 0; a < NF; ++a)
#pragma unroll
      for (int b = 0; b < NF; ++b) U[a][b] = ((a == b ? idt : S(0)) + S(g.self_adv) * U[a][b]) * act[a] * act[b];
  }
  // y_t = D_u^{-1} b_u(t), b_u = -(f - res) at the cell's u faces and p_{t+1},
  // from the rows (f - res) of u at slab t (ruv, the cell's faces) and of p (rpv)
  __device__ void u_solve_v(const T ruv[NF], T rpv, const CellG3<S>& cg, S y[NB]) const {
    S bf[NF], pb[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) bf[a] = S(-ruv[a]) * act[a];
    const S bp = S(-rpv);
    cg.proj(bf, pb);
    S gb = S(0);
#pragma unroll
    for (int a = 0; a < NF; ++a) gb += cg.gh[a] * bf[a];
#pragma unroll
    for (int a = 0; a < NF; ++a) y[a] = -pb[a] + cg.gh[a] * bp;
    y[NF] = gb + bp * cg.ig2;
  }
};

// The couplings U_t = I/dt + dAdv_loc(v_{t+1}) of every cell of the colour
// and every step, precomputed: each needs ~144 scattered loads of v around the
// cell, independent of the Thomas recurrence, which the thread-per-cell
// kernel otherwise issues twice per step inside its dependency chain.  Stored
// cell-fastest after the records (coalesced streaming loads in the solve).
// The colour's own faces of v_{t+1} are updated only after the solve's last
// use of U_t, and the stencil's other faces belong to other colours, so the
// values equal the ones the solve computed in place.  (Precomputing the
// residual-row loads as well -- y_t and the v-block right-hand side, 14
// loads per step -- measured no faster: the extra scratch traffic offset them.)
template <class T, class S>
__global__ void __launch_bounds__(128)
scgs3t_coupling_kernel(Geom g, const T* __restrict__ v, int colour, int ncell, S* __restrict__ ubuf) {
  pdl_wait();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (q >= ncell || t >= g.N) return;
  const ThomasCell<T, S> tc(g, colour, q);
  S U[NF][NF];
  tc.coupling(v + (size_t)(t + 1) * g.F, pick<S>(g.idt, g.idtf), U);
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int b = 0; b < NF; ++b) ubuf[((size_t)t * kThomasCpl + a * NF + b) * ncell + q] = U[a][b];
}

// Per-thread asynchronous copies (cp.async, sm_80+) that stage the global data
// one step of the Thomas kernel reads -- couplings, residual rows, records,
// state -- into the thread's own column of a two-stage shared-memory buffer one
// step ahead, so that no global load sits on the recurrence's dependency chain.
// Every thread copies and reads only its own column: the per-thread
// wait_group is the only synchronisation the buffer needs.
template <class E>
__device__ __forceinline__ void cpa(E* smem, const E* gmem) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8, "cp.async of 4 or 8 bytes");
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(E) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all groups but the most recent one complete
__device__ __forceinline__ void cpa_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

constexpr int kThomasThreads = 64;   // threads (cells) per CTA
constexpr int kStageS = kThomasRec;  // S values staged per step, at most (pass 2: a record)
constexpr int kStageT = 3 * NF + 3;  // T values staged per step, at most (pass 3: r.u, r.p, u, v, p, pbar)

template <class T, class S>
constexpr size_t scgs3t_smem_bytes() {
  return (size_t)2 * kThomasThreads * (kStageS * sizeof(S) + kStageT * sizeof(T));
}

template <class T, class S>
__global__ void __launch_bounds__(kThomasThreads)
scgs3t_colour_kernel(Geom g, State<T> x, CState<T> r, int colour, int ncell, const double* __restrict__ lm_dev,
                     S* __restrict__ zbuf) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncell) return;
  const int N = g.N;
  const S lm = S(lm_dev ? *lm_dev : g.lm);
  const S idt = pick<S>(g.idt, g.idtf);
  const ThomasCell<T, S> tc(g, colour, q);
  CellG3<S> cg;
  cg.init(g, tc.cl.i, tc.cl.j, tc.cl.k);
  auto rec = [&](int t, int e) -> S& { return zbuf[((size_t)t * kThomasRec + e) * ncell + q]; };
  const S* ubuf = zbuf + (size_t)kThomasRec * N * ncell;
  auto ucp = [&](int t, int e) -> const S* { return ubuf + ((size_t)t * kThomasCpl + e) * ncell + q; };
  // the thread's column of the staging buffers: [stage][element][thread]
  S* const stS = reinterpret_cast<S*>(smem_raw) + threadIdx.x;
  T* const stT = reinterpret_cast<T*>(smem_raw + (size_t)2 * kThomasThreads * kStageS * sizeof(S)) + threadIdx.x;
  auto sS = [&](int stage, int e) -> S& { return stS[(stage * kStageS + e) * kThomasThreads]; };
  auto sT = [&](int stage, int e) -> T& { return stT[(stage * kStageT + e) * kThomasThreads]; };
  auto stage_u = [&](int t, int stage) {
#pragma unroll
    for (int e = 0; e < kThomasCpl; ++e) cpa(&sS(stage, e), ucp(t, e));
  };
  auto stage_rup = [&](int t, int stage, int e0) {   // rows of u at the cell's faces and of p, slab t
    const T* ru = r.u + (size_t)t * g.F;
#pragma unroll
    for (int a = 0; a < NF; ++a) cpa(&sT(stage, e0 + a), ru + tc.fidx[a]);
    cpa(&sT(stage, e0 + NF), r.p + (size_t)t * g.C + tc.cc);
  };

  // ---- pass 1: ascending elimination ----------------------------------------
  // Slab s stages U_s, the rows of u and p at s (s < N) in S 0..35 / T 0..6,
  // and the rows of v and pbar at s (s >= 1) in T 7..13; the set-up consumes
  // slab 0, elimination step t slab t + 1.
  auto stage1 = [&](int s, int stage) {
    if (s < N) {
      stage_u(s, stage);
      stage_rup(s, stage, 0);
    }
    if (s >= 1) {
      const T* rv = r.v + (size_t)s * g.F;
#pragma unroll
      for (int a = 0; a < NF; ++a) cpa(&sT(stage, NB + a), rv + tc.fidx[a]);
      cpa(&sT(stage, NB + NF), r.pbar + (size_t)s * g.C + tc.cc);
    }
  };
  auto staged_y = [&](int stage, S y[NB]) {
    T ruv[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) ruv[a] = sT(stage, a);
    tc.u_solve_v(ruv, sT(stage, NF), cg, y);
  };
  auto staged_u = [&](int stage, S U[NF][NF]) {
#pragma unroll
    for (int a = 0; a < NF; ++a)
#pragma unroll
      for (int b = 0; b < NF; ++b) U[a][b] = sS(stage, a * NF + b);
  };

  // carried from block t-1: M = O_{t-1}^T X_{t-1} (faces), m = O_{t-1}^T z_{t-1};
  // from U_t (computed at block t-1): Sn = U_t^T P U_t, Rn = -U_t^T y_t
  S M[NF][NF], m[NF], Sn[NF][NF], Rn[NF];
  stage1(0, 0);
  cpa_commit();
  stage1(1, 1);
  cpa_commit();
  cpa_wait_prev();
  {
    S U[NF][NF], y[NB];
    staged_u(0, U);
    staged_y(0, y);
#pragma unroll
    for (int b = 0; b < NF; ++b) {
      S w[NF], pw[NF];
#pragma unroll
      for (int a = 0; a < NF; ++a) w[a] = U[a][b];
      cg.proj(w, pw);
#pragma unroll
      for (int a = 0; a < NF; ++a) Sn[a][b] = pw[a];   // P U column b (temporarily)
    }
    S PU[NF][NF];
#pragma unroll
    for (int a = 0; a < NF; ++a)
#pragma unroll
      for (int b = 0; b < NF; ++b) PU[a][b] = Sn[a][b];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
      for (int b = 0; b < NF; ++b) {
        S s = S(0);
#pragma unroll
        for (int c = 0; c < NF; ++c) s += U[c][a] * PU[c][b];
        Sn[a][b] = s;
      }
      S s = S(0);
#pragma unroll
      for (int c = 0; c < NF; ++c) s += U[c][a] * y[c];
      Rn[a] = -s;
      m[a] = S(0);
#pragma unroll
      for (int b = 0; b < NF; ++b) M[a][b] = S(0);
    }
  }
  for (int t = 0; t < N; ++t) {
    const int tv = t + 1;
    const int cur = tv & 1;
    if (tv + 1 <= N) stage1(tv + 1, (tv + 1) & 1);   // the stage slab t - 1 used
    cpa_commit();
    cpa_wait_prev();                                   // slab tv has landed
    // pivot block of v_tv
    S A[NF][NF], B[NF][NB], qv[NB];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
      for (int b = 0; b < NF; ++b) {
        S v = Sn[a][b] - M[a][b];
        if (tv < N) v += ((a == b ? cg.act[a] : S(0)) - cg.gh[a] * cg.g[b]) * idt * idt;
        if (a == b) v += cg.act[a] > S(0) ? ((tv < N ? pick<S>(g.a, g.af) : S(0)) + lm) : S(1);
        A[a][b] = v;
      }
      B[a][NF] = S(-sT(cur, NB + a)) * tc.act[a] + Rn[a] - m[a];
    }
    qv[NF] = S(-sT(cur, NB + NF));
    // coupling to v_{tv+1}: O = -P U_tv / dt, and the next block's Sn, Rn
    if (tv < N) {
      S U[NF][NF], y[NB];
      staged_u(cur, U);
      staged_y(cur, y);
#pragma unroll
      for (int a = 0; a < NF; ++a) B[a][NF] += idt * cg.act[a] * y[a];
      S PU[NF][NF];
#pragma unroll
      for (int b = 0; b < NF; ++b) {
        S w[NF], pw[NF];
#pragma unroll
        for (int a = 0; a < NF; ++a) w[a] = U[a][b];
        cg.proj(w, pw);
#pragma unroll
        for (int a = 0; a < NF; ++a) {
          PU[a][b] = pw[a];
          B[a][b] = -idt * pw[a];
        }
      }
#pragma unroll
      for (int a = 0; a < NF; ++a) {
#pragma unroll
        for (int b = 0; b < NF; ++b) {
          S s = S(0);
#pragma unroll
          for (int c = 0; c < NF; ++c) s += U[c][a] * PU[c][b];
          Sn[a][b] = s;
        }
        S s = S(0);
#pragma unroll
        for (int c = 0; c < NF; ++c) s += U[c][a] * y[c];
        Rn[a] = -s;
      }
    } else {
#pragma unroll
      for (int a = 0; a < NF; ++a)
#pragma unroll
        for (int b = 0; b < NF; ++b) B[a][b] = S(0);
    }
#pragma unroll
    for (int c = 0; c < NF; ++c) qv[c] = S(0);
    const S gam = shift_sym6(A, cg);
    S Y[NB];
    S O[NF][NF];
#pragma unroll
    for (int a = 0; a < NF; ++a)
#pragma unroll
      for (int b = 0; b < NF; ++b) O[a][b] = B[a][b];
    saddle_solve6<S, NB>(A, cg.g, B, qv, Y);
    Y[NF] += gam * qv[NF];
    // record Z_t = (X, multipliers) and z_t
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
      for (int b = 0; b < NF; ++b) rec(t, a * NF + b) = B[a][b];
      rec(t, NF * NF + a) = Y[a];
      rec(t, NF * NF + NF + a) = B[a][NF];
    }
    rec(t, NF * NF + 2 * NF) = Y[NF];
    // carried into the next pivot: M = O^T X, m = O^T z (faces)
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
      for (int b = 0; b < NF; ++b) {
        S s = S(0);
#pragma unroll
        for (int c = 0; c < NF; ++c) s += O[c][a] * B[c][b];
        M[a][b] = s;
      }
      S s = S(0);
#pragma unroll
      for (int c = 0; c < NF; ++c) s += O[c][a] * B[c][NF];
      m[a] = s;
    }
  }

  // ---- pass 2: descending substitution, x_t overwrites z_t -------------------
  // Step i stages the record of block t = N - 1 - i (written in pass 1 by this
  // thread; the fence orders those stores before the copies that read them).
  __threadfence_block();
  auto stage2 = [&](int t, int stage) {
#pragma unroll
    for (int e = 0; e < kThomasRec; ++e) cpa(&sS(stage, e), &rec(t, e));
  };
  {
    S xn[NF];
    stage2(N - 1, 0);
    cpa_commit();
    if (N >= 2) stage2(N - 2, 1);
    cpa_commit();
    cpa_wait_prev();
#pragma unroll
    for (int a = 0; a < NF; ++a) xn[a] = sS(0, NF * NF + NF + a);
    for (int t = N - 2; t >= 0; --t) {
      const int i = N - 1 - t, cur = i & 1;
      if (t >= 1) stage2(t - 1, (i + 1) & 1);
      cpa_commit();
      cpa_wait_prev();
      S xt[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        S v = sS(cur, NF * NF + NF + a);
#pragma unroll
        for (int b = 0; b < NF; ++b) v -= (a < NF ? sS(cur, a * NF + b) : sS(cur, NF * NF + b)) * xn[b];
        xt[a] = v;
      }
#pragma unroll
      for (int a = 0; a < NB; ++a) rec(t, NF * NF + NF + a) = xt[a];
#pragma unroll
      for (int a = 0; a < NF; ++a) xn[a] = xt[a];
    }
  }

  // ---- pass 3: u blocks from the v solution, x += omega delta ---------------
  // Step t stages U_t (S 0..35), the v-block solution x_t (S 36..42), the rows
  // of u and p at t (T 0..6) and the state it updates: u_t and v_{t+1} at the
  // cell's faces (T 7..18), p_t and pbar_{t+1} at the cell (T 19, 20).  Only
  // this thread writes those entries, each after its own copy has landed.
  __threadfence_block();
  auto stage3 = [&](int t, int stage) {
    stage_u(t, stage);
#pragma unroll
    for (int a = 0; a < NB; ++a) cpa(&sS(stage, kThomasCpl + a), &rec(t, NF * NF + NF + a));
    stage_rup(t, stage, 0);
    const T* fu = x.u + (size_t)t * g.F;
    const T* fv = x.v + (size_t)(t + 1) * g.F;
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      cpa(&sT(stage, NB + a), fu + tc.fidx[a]);
      cpa(&sT(stage, NB + NF + a), fv + tc.fidx[a]);
    }
    cpa(&sT(stage, NB + 2 * NF), x.p + (size_t)t * g.C + tc.cc);
    cpa(&sT(stage, NB + 2 * NF + 1), x.pbar + (size_t)(t + 1) * g.C + tc.cc);
  };
  const T om = pick<T>(g.omega, g.omegaf);
  S xv0[NF];
#pragma unroll
  for (int a = 0; a < NF; ++a) xv0[a] = S(0);
  stage3(0, 0);
  cpa_commit();
  for (int t = 0; t < N; ++t) {
    const int cur = t & 1;
    if (t + 1 < N) stage3(t + 1, (t + 1) & 1);
    cpa_commit();
    cpa_wait_prev();
    S U[NF][NF], y[NB], xv1[NB];
    staged_u(cur, U);
    staged_y(cur, y);
#pragma unroll
    for (int a = 0; a < NB; ++a) xv1[a] = sS(cur, kThomasCpl + a);
    S w[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      S v = S(0);
#pragma unroll
      for (int b = 0; b < NF; ++b) v -= U[a][b] * xv1[b];
      if (t >= 1) v += idt * cg.act[a] * xv0[a];
      w[a] = v;
    }
    S pw[NF];
    cg.proj(w, pw);
    S gw = S(0);
#pragma unroll
    for (int a = 0; a < NF; ++a) gw += cg.gh[a] * w[a];
    T* fu = x.u + (size_t)t * g.F;
    T* fv = x.v + (size_t)(t + 1) * g.F;
#pragma unroll
    for (int a = 0; a < NF; ++a)
      if (tc.act[a] > S(0)) {
        const int f = tc.fidx[a];
        fu[f] = sT(cur, NB + a) + om * T(y[a] - pw[a]);
        fv[f] = sT(cur, NB + NF + a) + om * T(xv1[a]);
      }
    x.p[(size_t)t * g.C + tc.cc] = sT(cur, NB + 2 * NF) + om * T(y[NF] + gw);
    x.pbar[(size_t)(t + 1) * g.C + tc.cc] = sT(cur, NB + 2 * NF + 1) + om * T(xv1[NF]);
#pragma unroll
    for (int a = 0; a < NF; ++a) xv0[a] = xv1[a];
  }
}

// ---------------------------------------------------------------------------
// transfers (Sec. 4.3 with a third axis): R = mean of the 8 children (cells) /
// the 4 coincident fine faces (faces); P = trilinear, faces linear along the
// normal and (3/4, 1/4) across, clamped at walls.  Time modes as the 2D
// kernels (0 same slabs, 1 points, 2 intervals, 3 targets).
// ---------------------------------------------------------------------------
template <class Tc, class RS>
__device__ __forceinline__ Tc in_time_r(RS rs, int tmode, int t, int nt) {
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
}

template <class Tf, class Tc>
__global__ void restrict3_kernel(Geom gf, Geom gc, int nt_face, int nt_cell, const Tf* __restrict__ sf,
                                 const Tf* __restrict__ sc_cells, Tc* df, Tc* dc_cells, Tc* df2, Tc* dc2, int tmode) {
  pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nfaces = (size_t)nt_face * gc.F;
  const size_t ncells = (size_t)nt_cell * gc.C;
  if (e < nfaces) {
    const int t = (int)(e / gc.F);
    const int f = (int)(e - (size_t)t * gc.F);
    int K, J, I;
    const int axis = face_coords(gc, f, K, J, I);
    const bool slot = !gc.periodic || is_face(gc, axis, K, J, I);   // the unused periodic slot stays 0
    auto rs = [&](int tf) -> Tc {
      if (!slot) return Tc(0);
      const Tf* s = sf + (size_t)tf * gf.F;
      Tc acc = Tc(0);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          int idx;
          if (axis == 0) idx = xf(gf, 2 * K + a, 2 * J + b, 2 * I);
          else if (axis == 1) idx = yf(gf, 2 * K + a, 2 * J, 2 * I + b);
          else idx = zf(gf, 2 * K, 2 * J + a, 2 * I + b);
          acc += Tc(s[idx]);
        }
      return Tc(0.25) * acc;
    };
    const Tc val = in_time_r<Tc>(rs, tmode, t, nt_face);
    df[e] = val;
    if (df2) df2[e] = val;
  } else if (e < nfaces + ncells) {
    const size_t ec = e - nfaces;
    const int t = (int)(ec / gc.C);
    const int c = (int)(ec - (size_t)t * gc.C);
    const int I = c % gc.nx, r = c / gc.nx, J = r % gc.ny, K = r / gc.ny;
    auto rs = [&](int tf) -> Tc {
      const Tf* s = sc_cells + (size_t)tf * gf.C;
      Tc acc = Tc(0);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int d = 0; d < 2; ++d) acc += Tc(s[cid(gf, 2 * K + a, 2 * J + b, 2 * I + d)]);
      return Tc(0.125) * acc;
    };
    const Tc val = in_time_r<Tc>(rs, tmode, t, nt_cell);
    dc_cells[ec] = val;
    if (dc2) dc2[ec] = val;
  }
}

// (3/4, 1/4) neighbours of fine cell k among nc coarse cells: clamped at a
// wall, wrapped on a periodic axis
__device__ __forceinline__ void cell_interp3(int k, int nc, int& a, int& b, bool periodic = false) {
  a = k >> 1;
  b = (k & 1) ? a + 1 : a - 1;
  if (periodic) b = b < 0 ? b + nc : (b > nc - 1 ? b - nc : b);
  else b = b < 0 ? 0 : (b > nc - 1 ? nc - 1 : b);
}

template <class Tf, class Tc>
__global__ void prolong3_correct_kernel(Geom gf, Geom gc, int nt_face, int nt_cell, int t0_face, int t0_cell, Tf* ff,
                                        Tf* fc, const Tc* __restrict__ cnf, const Tc* __restrict__ cof,
                                        const Tc* __restrict__ cnc, const Tc* __restrict__ coc,
                                        const double* undo_if_rose, int tmode) {
  pdl_wait();
  using W = typename std::conditional<(sizeof(Tf) == 8 || sizeof(Tc) == 8), double, float>::type;
  W sgn = W(1);
  if (undo_if_rose) {
    if (undo_if_rose[1] <= undo_if_rose[0]) return;
    sgn = W(-1);
  }
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nfaces = (size_t)nt_face * gf.F;
  const size_t ncells = (size_t)nt_cell * gf.C;
  auto in_time = [&](auto ps, int t) -> W {
    if (tmode == 0) return ps(t);
    if (tmode == 2) return ps(t >> 1);
    if ((t & 1) == 0) return ps(t >> 1);
    return W(0.5) * (ps(t >> 1) + ps((t >> 1) + 1));
  };
  if (e < nfaces) {
    const int t = (int)(e / gf.F) + t0_face;
    const int f = (int)(e - (size_t)(t - t0_face) * gf.F);
    int k, j, i;
    const int axis = face_coords(gf, f, k, j, i);
    if (gf.periodic && !is_face(gf, axis, k, j, i)) return;
    // per axis (k, j, i): two coarse indices and weights
    int ca[3], cb[3];
    W wa[3], wb[3];
    const int fine[3] = {k, j, i};
    const int nce[3] = {gc.nz, gc.ny, gc.nx};
    const int normal = 2 - axis;   // array axis of the face normal (x -> i)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d == normal) {
        ca[d] = fine[d] >> 1;
        cb[d] = (fine[d] & 1) ? ca[d] + 1 : ca[d];
        wb[d] = (fine[d] & 1) ? W(0.5) : W(0);
        wa[d] = W(1) - wb[d];
      } else {
        cell_interp3(fine[d], nce[d], ca[d], cb[d], gf.periodic != 0);
        wa[d] = W(0.75);
        wb[d] = W(0.25);
      }
    }
    auto ps = [&](int tc) -> W {
      const Tc* n = cnf + (size_t)tc * gc.F;
      const Tc* o = cof + (size_t)tc * gc.F;
      W val = W(0);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int K = a ? cb[0] : ca[0], J = b ? cb[1] : ca[1], I = c ? cb[2] : ca[2];
            const W w = (a ? wb[0] : wa[0]) * (b ? wb[1] : wa[1]) * (c ? wb[2] : wa[2]);
            if (w == W(0)) continue;
            const int idx = axis == 0 ? xf(gc, K, J, I) : (axis == 1 ? yf(gc, K, J, I) : zf(gc, K, J, I));
            val += w * (W(n[idx]) - W(o[idx]));
          }
      return val;
    };
    ff[(size_t)t * gf.F + f] += Tf(sgn * in_time(ps, t));
  } else if (e < nfaces + ncells) {
    const size_t ec = e - nfaces;
    const int t = (int)(ec / gf.C) + t0_cell;
    const int c = (int)(ec - (size_t)(t - t0_cell) * gf.C);
    const int i = c % gf.nx, r = c / gf.nx, j = r % gf.ny, k = r / gf.ny;
    int ka, kb, ja, jb, ia, ib;
    cell_interp3(k, gc.nz, ka, kb, gf.periodic != 0);
    cell_interp3(j, gc.ny, ja, jb, gf.periodic != 0);
    cell_interp3(i, gc.nx, ia, ib, gf.periodic != 0);
    auto ps = [&](int tc) -> W {
      const Tc* n = cnc + (size_t)tc * gc.C;
      const Tc* o = coc + (size_t)tc * gc.C;
      W val = W(0);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            const int idx = cid(gc, a ? kb : ka, b ? jb : ja, d ? ib : ia);
            const W w = (a ? W(0.25) : W(0.75)) * (b ? W(0.25) : W(0.75)) * (d ? W(0.25) : W(0.75));
            val += w * (W(n[idx]) - W(o[idx]));
          }
      return val;
    };
    fc[(size_t)t * gf.C + c] += Tf(sgn * in_time(ps, t));
  }
}

// u_raw_t = (v_{t+1} - v_t)/dt + Adv(v_{t+1}), t = 0..N-1   (Appendix A)
template <class T>
__global__ void kkt_force_rhs3_kernel(Geom g, const T* __restrict__ v, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (e >= g.F || t >= g.N) return;
  const T* vn = v + (size_t)(t + 1) * g.F;
  const T* vt = v + (size_t)t * g.F;
  int k, j, i;
  const int axis = face_coords(g, e, k, j, i);
  T val = T(0);
  if (is_face(g, axis, k, j, i))
    val = (vn[e] - vt[e]) * pick<T>(g.idt, g.idtf) + T(g.self_adv) * adv(g, vn, axis, k, j, i);
  out[(size_t)t * g.F + e] = val;
}

// g_raw_t = r(u_{t-1}/dt + dAdv(v_t)^T u_{t-1} - u_t/dt [t<N]) + dens_t, t = 1..N
template <class T>
__global__ void kkt_grad_rhs3_kernel(Geom g, const T* __restrict__ v, const T* __restrict__ u,
                                     const T* __restrict__ dens, double r, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y + 1;
  if (e >= g.F || t > g.N) return;
  const T* vt = v + (size_t)t * g.F;
  const T* um = u + (size_t)(t - 1) * g.F;
  int k, j, i;
  const int axis = face_coords(g, e, k, j, i);
  T val = T(0);
  if (is_face(g, axis, k, j, i)) {
    T s = um[e] * pick<T>(g.idt, g.idtf);
    if (g.self_adv) s += jtu(g, vt, um, axis, k, j, i);
    if (t < g.N) s -= u[(size_t)t * g.F + e] * pick<T>(g.idt, g.idtf);
    val = T(r) * s + dens[(size_t)t * g.F + e];
  }
  out[(size_t)t * g.F + e] = val;
}

template <class... KArgs, class... Args>
void launch_pdl3(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

inline unsigned blocks3(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers (called by the dimension-generic launchers when g.dim == 3)
// ---------------------------------------------------------------------------
// pass A of the two-pass rows on levels of at least this many faces.  Every
// level qualifies: on the small levels, and on the fp64 coarsest level at
// GB300's low fp64 rate, the inline gathers cost more than the three extra
// launches (measured inline: ~60-100 us per colour residual on 16^3 .. 4^3).
constexpr int kLambMinFaces = 0;

size_t lamb3_scratch_bytes(const Geom& g, size_t tsize) {
  return g.F < kLambMinFaces ? 0 : (size_t)(g.N + 1) * g.F * 5 * tsize;
}

// the scratch of a whole hierarchy: the largest level's need (the finest in
// its type, or the fp64 coarsest level of an fp32 hierarchy)
size_t lamb3_scratch_bytes_max(const Geom& finest, size_t tsize, const Geom& coarsest, size_t csize) {
  const size_t a = lamb3_scratch_bytes(finest, tsize), b = lamb3_scratch_bytes(coarsest, csize);
  return a > b ? a : b;
}

// pass A into the scratch (AB4 slices then the Adv slices); false: inline form
template <class T>
bool lamb3_pass_a(const Geom& g, CState<T> x, void* scratch, size_t bytes, cudaStream_t st, AB4<T>** ab,
                  T** advb) {
  if (!scratch || g.F < kLambMinFaces || bytes < lamb3_scratch_bytes(g, sizeof(T))) return false;
  *ab = reinterpret_cast<AB4<T>*>(scratch);
  *advb = reinterpret_cast<T*>(*ab + (size_t)(g.N + 1) * g.F);
  const int nfx = (g.nx + 1) * g.ny * g.nz, nfy = g.nx * (g.ny + 1) * g.nz, nfz = g.nx * g.ny * (g.nz + 1);
  launch_pdl3(lamb3_terms_kernel<T, 0>, dim3(blocks3(nfx, 128), g.N + 1), dim3(128), 0, st, g, x.v, x.u, *ab, *advb);
  launch_pdl3(lamb3_terms_kernel<T, 1>, dim3(blocks3(nfy, 128), g.N + 1), dim3(128), 0, st, g, x.v, x.u, *ab, *advb);
  launch_pdl3(lamb3_terms_kernel<T, 2>, dim3(blocks3(nfz, 128), g.N + 1), dim3(128), 0, st, g, x.v, x.u, *ab, *advb);
  return true;
}

template <class T>
int launch_nso_residual3(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, T sf, T sr,
                         cudaStream_t st, double* sq, const double* only_if_undone, RedScratch rs, void* lamb,
                         size_t lamb_bytes) {
  const int n = g.F > g.C ? g.F : g.C;
  AB4<T>* ab = nullptr;
  T* advb = nullptr;
  if (lamb3_pass_a(g, x, lamb, lamb_bytes, st, &ab, &advb)) {
    launch_pdl3(nso_residual3_kernel<T, true>, dim3(blocks3(n, 128), g.N + 1), dim3(128), 0, st, g, x, z, res, out,
                sf, sr, sq, rs, only_if_undone, (const AB4<T>*)ab, (const T*)advb);
    return 4;
  }
  launch_pdl3(nso_residual3_kernel<T, false>, dim3(blocks3(n, 128), g.N + 1), dim3(128), 0, st, g, x, z, res, out,
              sf, sr, sq, rs, only_if_undone, (const AB4<T>*)nullptr, (const T*)nullptr);
  return 1;
}

size_t nso_residual3_blocks(const Geom& g) {
  const int n = g.F > g.C ? g.F : g.C;
  return (size_t)blocks3(n, 128) * (g.N + 1);
}

template <class T>
int launch_nso_residual3_colour(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, int colour,
                                cudaStream_t st, const double* only_if_undone, void* lamb, size_t lamb_bytes) {
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int ncx = (g.nx - px + 1) / 2, ncy = (g.ny - py + 1) / 2, ncz = (g.nz - pz + 1) / 2;
  const int n = ncz * ncy * (g.nx + 1) + ncz * (g.ny + 1) * ncx + (g.nz + 1) * ncy * ncx + ncx * ncy * ncz;
  AB4<T>* ab = nullptr;
  T* advb = nullptr;
  if (lamb3_pass_a(g, x, lamb, lamb_bytes, st, &ab, &advb)) {
    launch_pdl3(nso_residual3_colour_kernel<T, true>, dim3(blocks3(n, 128), g.N + 1), dim3(128), 0, st, g, x, z, res,
                out, px, py, pz, only_if_undone, (const AB4<T>*)ab, (const T*)advb);
    return 4;
  }
  launch_pdl3(nso_residual3_colour_kernel<T, false>, dim3(blocks3(n, 128), g.N + 1), dim3(128), 0, st, g, x, z, res,
              out, px, py, pz, only_if_undone, (const AB4<T>*)nullptr, (const T*)nullptr);
  return 1;
}

size_t scgs3_smem_bytes(int N, size_t tsize) { return scgs3_cell_floats(N) * tsize; }

// cells per CTA: as many as fit the opt-in shared memory, at most 8 (one warp each)
static int scgs3_cells_per_block(int N, size_t ssize) {
  static std::once_flag once;
  static int optin = 0;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    optin -= 1024;   // the kernel's static shared memory
  });
  int cpb = (int)((size_t)optin / scgs3_smem_bytes(N, ssize));
  return cpb > 8 ? 8 : cpb;
}

template <class T, class S>
static int launch_scgs3_ts(const Geom& g, State<T> x, CState<T> r, int colour, const double* lm_dev,
                           cudaStream_t st, void* scratch) {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncGetAttributes(&fa, (const void*)scgs3_colour_kernel<T, S>);
    cudaFuncSetAttribute((const void*)scgs3_colour_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin - (int)fa.sharedSizeBytes);
  });
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int ncell = ((g.nx - px + 1) / 2) * ((g.ny - py + 1) / 2) * ((g.nz - pz + 1) / 2);
  if (ncell == 0) return 0;
  const int cpb = scgs3_cells_per_block(g.N, sizeof(S));
  if (cpb < 1) return 0;   // refused at problem creation (scgs_smem_bytes)
  const size_t smem = (size_t)cpb * scgs3_smem_bytes(g.N, sizeof(S));
  const int threads = 32 * cpb < 64 ? 64 : 32 * cpb;
  S* ubuf = static_cast<S*>(scratch);
  if (ubuf)   // (a coarser level's colour fits the finest level's scratch)
    launch_pdl3(scgs3t_coupling_kernel<T, S>, dim3((ncell + 127) / 128, g.N), dim3(128), 0, st, g, (const T*)x.v,
                colour, ncell, ubuf);
  launch_pdl3(scgs3_colour_kernel<T, S>, dim3((ncell + cpb - 1) / cpb), dim3(threads), smem, st, g, x, r, colour,
              ncell, cpb, lm_dev, (const S*)ubuf);
  return ubuf ? 2 : 1;
}

// Colours with at least kThomasMinCells cells run the thread-per-cell block
// Thomas kernel (given its scratch); smaller ones the cyclic reduction, whose
// critical path is log N rather than N block steps.
constexpr int kThomasMinCells = 16384;

size_t scgs3_thomas_scratch_bytes(const Geom& g, size_t ssize) {
  const size_t ncell = (size_t)((g.nx + 1) / 2) * ((g.ny + 1) / 2) * ((g.nz + 1) / 2);
  return (size_t)(kThomasRec + kThomasCpl) * g.N * ncell * ssize;   // records, then couplings
}

template <class T, class S>
static void launch_scgs3t(const Geom& g, State<T> x, CState<T> r, int colour, const double* lm_dev, void* scratch,
                          cudaStream_t st) {
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int ncell = ((g.nx - px + 1) / 2) * ((g.ny - py + 1) / 2) * ((g.nz - pz + 1) / 2);
  S* zbuf = static_cast<S*>(scratch);
  launch_pdl3(scgs3t_coupling_kernel<T, S>, dim3((ncell + 127) / 128, g.N), dim3(128), 0, st, g, (const T*)x.v,
              colour, ncell, zbuf + (size_t)kThomasRec * g.N * ncell);
  constexpr size_t smem = scgs3t_smem_bytes<T, S>();
  static std::once_flag once;
  std::call_once(once, [] {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute((const void*)scgs3t_colour_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  });
  launch_pdl3(scgs3t_colour_kernel<T, S>, dim3((ncell + kThomasThreads - 1) / kThomasThreads), dim3(kThomasThreads),
              smem, st, g, x, r, colour, ncell, lm_dev, zbuf);
}

template <class T>
int launch_scgs3_colour(const Geom& g, State<T> x, CState<T> r, int colour, bool solve_fp32, cudaStream_t st,
                         const double* lm_dev, void* scratch) {
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int ncell = ((g.nx - px + 1) / 2) * ((g.ny - py + 1) / 2) * ((g.nz - pz + 1) / 2);
  if (scratch && ncell >= kThomasMinCells) {
    if (solve_fp32) launch_scgs3t<T, float>(g, x, r, colour, lm_dev, scratch, st);
    else launch_scgs3t<T, T>(g, x, r, colour, lm_dev, scratch, st);
    return 2;   // the couplings, then the Thomas solve
  }
  if (solve_fp32) return launch_scgs3_ts<T, float>(g, x, r, colour, lm_dev, st, scratch);
  return launch_scgs3_ts<T, T>(g, x, r, colour, lm_dev, st, scratch);
}

template <class Tf, class Tc>
void launch_restrict3(const Geom& gf, const Geom& gc, CState<Tf> s, State<Tc> d, State<Tc> d2, cudaStream_t st) {
  const bool in_time = gc.N != gf.N;
  const size_t nv = (size_t)(gc.N + 1) * gc.F + (size_t)(gc.N + 1) * gc.C;
  launch_pdl3(restrict3_kernel<Tf, Tc>, dim3(blocks3(nv, 256)), dim3(256), 0, st, gf, gc, gc.N + 1, gc.N + 1, s.v,
              s.pbar, d.v, d.pbar, d2.v, d2.pbar, in_time ? 1 : 0);
  const size_t nu = (size_t)gc.N * gc.F + (size_t)gc.N * gc.C;
  launch_pdl3(restrict3_kernel<Tf, Tc>, dim3(blocks3(nu, 256)), dim3(256), 0, st, gf, gc, gc.N, gc.N, s.u, s.p, d.u,
              d.p, d2.u, d2.p, in_time ? 2 : 0);
}

template <class Tf, class Tc>
void launch_restrict3_faces(const Geom& gf, const Geom& gc, int nt, const Tf* s, Tc* d, cudaStream_t st) {
  const bool in_time = gc.N != gf.N;
  const int ntc = in_time ? nt / 2 : nt;
  const size_t n = (size_t)ntc * gc.F;
  if (n == 0) return;
  launch_pdl3(restrict3_kernel<Tf, Tc>, dim3(blocks3(n, 256)), dim3(256), 0, st, gf, gc, ntc, 0, s, (const Tf*)nullptr,
              d, (Tc*)nullptr, (Tc*)nullptr, (Tc*)nullptr, in_time ? 3 : 0);
}

template <class Tf, class Tc>
void launch_prolong3_correct(const Geom& gf, const Geom& gc, State<Tf> f, CState<Tc> cn, CState<Tc> co,
                             cudaStream_t st, const double* undo_if_rose) {
  const bool in_time = gc.N != gf.N;
  // v and pbar from slab 1 (v_0 fixed, pbar_0 unused)
  const size_t nv = (size_t)gf.N * gf.F + (size_t)gf.N * gf.C;
  launch_pdl3(prolong3_correct_kernel<Tf, Tc>, dim3(blocks3(nv, 256)), dim3(256), 0, st, gf, gc, gf.N, gf.N, 1, 1,
              f.v, f.pbar, cn.v, co.v, cn.pbar, co.pbar, undo_if_rose, in_time ? 1 : 0);
  const size_t nu = (size_t)gf.N * gf.F + (size_t)gf.N * gf.C;
  launch_pdl3(prolong3_correct_kernel<Tf, Tc>, dim3(blocks3(nu, 256)), dim3(256), 0, st, gf, gc, gf.N, gf.N, 0, 0,
              f.u, f.p, cn.u, co.u, cn.p, co.p, undo_if_rose, in_time ? 2 : 0);
}

template <class T>
void launch_kkt_force_rhs3(const Geom& g, const T* v, T* out, cudaStream_t st) {
  kkt_force_rhs3_kernel<T><<<dim3(blocks3(g.F, 128), g.N), 128, 0, st>>>(g, v, out);
}

template <class T>
void launch_kkt_grad_rhs3(const Geom& g, const T* v, const T* u, const T* dens, double r, T* out, cudaStream_t st) {
  kkt_grad_rhs3_kernel<T><<<dim3(blocks3(g.F, 128), g.N), 128, 0, st>>>(g, v, u, dens, r, out);
}

#define STC3_INST_T(T)                                                                                         \
  template int launch_nso_residual3<T>(const Geom&, CState<T>, const T*, CState<T>, State<T>, T, T,           \
                                       cudaStream_t, double*, const double*, RedScratch, void*, size_t);       \
  template int launch_nso_residual3_colour<T>(const Geom&, CState<T>, const T*, CState<T>, State<T>, int,     \
                                              cudaStream_t, const double*, void*, size_t);                    \
  template int launch_scgs3_colour<T>(const Geom&, State<T>, CState<T>, int, bool, cudaStream_t,             \
                                       const double*, void*);                                                 \
  template void launch_kkt_force_rhs3<T>(const Geom&, const T*, T*, cudaStream_t);                            \
  template void launch_kkt_grad_rhs3<T>(const Geom&, const T*, const T*, const T*, double, T*, cudaStream_t);
STC3_INST_T(float)
STC3_INST_T(double)

#define STC3_INST_TT(Tf, Tc)                                                                                   \
  template void launch_restrict3<Tf, Tc>(const Geom&, const Geom&, CState<Tf>, State<Tc>, State<Tc>,          \
                                         cudaStream_t);                                                       \
  template void launch_restrict3_faces<Tf, Tc>(const Geom&, const Geom&, int, const Tf*, Tc*, cudaStream_t);  \
  template void launch_prolong3_correct<Tf, Tc>(const Geom&, const Geom&, State<Tf>, CState<Tc>, CState<Tc>, \
                                                cudaStream_t, const double*);
STC3_INST_TT(float, float)
STC3_INST_TT(double, double)
STC3_INST_TT(float, double)
STC3_INST_TT(double, float)

}  // namespace stc
