// Launchers of the CUDA kernels of libstc (host-callable, internal).
#pragma once

#include "stc_internal.cuh"

namespace stc {

// thread-local message returned by stc_last_error()
void set_last_error(const char* msg);

// --- NSO (nso_kernels.cu) ---------------------------------------------------
// out = sf * f(x) + sr * res.  sq (optional): += sum of squares of out (fp64,
// summed in block order through rs, which needs nso_residual_blocks(g) partials).
// only_if_undone (optional, a guard's {before, after} norms): skip unless the
// guarded coarse-grid correction was undone (after > before or NaN).
template <class T>
int launch_nso_residual(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, T sf, T sr,
                        cudaStream_t st, double* sq = nullptr, const double* only_if_undone = nullptr,
                        RedScratch rs = RedScratch{}, void* lamb = nullptr, size_t lamb_bytes = 0);
// blocks of a launch_nso_residual launch (the RedScratch capacity its sq needs)
size_t nso_residual_blocks(const Geom& g);
size_t nso_residual3_blocks(const Geom& g);
// most blocks of the other reductions (sumsq, diff_sumsq; misfit_dot uses fewer)
constexpr unsigned kReduceMaxBlocks = 1216;
// out = f - res at the faces and cells one SCGS colour reads (other entries untouched);
// only_if_undone as in launch_nso_residual
template <class T>
int launch_nso_residual_colour(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, int colour,
                               cudaStream_t st, const double* only_if_undone = nullptr, void* lamb = nullptr,
                               size_t lamb_bytes = 0);
// lm_dev (optional): device fp64 Levenberg-Marquardt shift of the v blocks, else g.lm;
// scratch3 (3D, optional): scgs3_thomas_scratch_bytes of the finest level, which
// lets large colours run the thread-per-cell block Thomas kernel
template <class T>
int launch_scgs_colour(const Geom& g, State<T> x, CState<T> r, int colour, bool solve_fp32, cudaStream_t st,
                        const double* lm_dev = nullptr, void* scratch3 = nullptr);
size_t scgs_smem_bytes(int N, size_t tsize);
int colour_extent(int n, int parity);
template <class Tf, class Tc>
void launch_restrict(const Geom& gf, const Geom& gc, CState<Tf> s, State<Tc> d, State<Tc> d2, cudaStream_t st);
template <class Tf, class Tc>
void launch_restrict_faces(const Geom& gf, const Geom& gc, int nt, const Tf* s, Tc* d, cudaStream_t st);
// f += P(cn - co); with undo_if_rose = a guard's {before, after} norms, instead
// f -= P(cn - co) when after > before (or NaN), and nothing otherwise.
template <class Tf, class Tc>
void launch_prolong_correct(const Geom& gf, const Geom& gc, State<Tf> f, CState<Tc> cn, CState<Tc> co,
                            cudaStream_t st, const double* undo_if_rose = nullptr);
template <class T>
void launch_absmax(const T* a, size_t n, double* out, int* err, cudaStream_t st);
// *out += sum of a_e^2 (fp64, block order through rs; at most kReduceMaxBlocks blocks)
template <class T>
void launch_sumsq(const T* a, size_t n, double* out, cudaStream_t st, RedScratch rs);
template <class T>
void launch_remove_mean(T* a, int count, int C, cudaStream_t st);
template <class Ts, class Td>
void launch_convert(const Ts* s, Td* d, size_t n, cudaStream_t st);

// --- advection (advect_kernels.cu) ------------------------------------------
constexpr int kMaxClusterCTAs = 16;   // the sweeps run on one cluster of 16 (non-portable) or 8 CTAs
// cluster size of the advection sweeps on this device: 16 when a 16-CTA cluster
// of the sweep kernels can be scheduled, else 8 (decided once per process)
int advect_cluster_ctas();
constexpr int kAdvThreads = 512;
constexpr int kTaylorKmaxLimit = 256;   // largest taylor_kmax (size of the sweeps' dt/k tables)
constexpr int kAdvMaxCellsPerThread = 8;

// rho[0] given; writes rho[1..N] and K[0..N-1] (Taylor orders).  vel: N face slabs.
template <class T>
cudaError_t launch_taylor_forward(const Geom& g, const T* vel, T* rho, int* K, double thresh, int kmax, int* err,
                                  cudaStream_t st);
// Backward adjoint sweep (Eq. KKTPO): mu_{s-1} = T_s^T mu_s - m_s, mu_{N-1} = -m_N;
// out_s = alpha * base_s + beta * (dA[rho_s, v_s]/dv)^T mu_s for s = 1..N-1.
// s_end = 1: steps N-1..1 (the AO sweep; v_0 is data).  s_end = 0 also runs step
// 0: out_0 and, into mu_m1 (C entries, may be null), T_0^T mu_0 - m_0 (the
// adjoint density of rho_0, for chaining simulation segments); mu_0 stays mu_0.
// A Taylor order outside 1..kmax sets DEV_TAYLOR_KMAX in *err (may be null).
template <class T>
cudaError_t launch_taylor_adjoint(const Geom& g, const T* vel, const T* rho, const int* K, const double* mterm,
                                  T* mu, const T* base, T alpha, T beta, T* out, T* powers, int kmax,
                                  int* err, cudaStream_t st, int s_end = 1, T* mu_m1 = nullptr);
// doubles of launch_metric's tmp1 for C cells and the given levels
size_t metric_tmp1_doubles(size_t C, int levels);
// m_s = c * sum_l G_l^T G_l (rho_s - rho*_s) (fp64) into mterm slab s.
template <class T>
void launch_metric(const Geom& g, const T* rho_s, const double* star, double c, int levels, double sigma0,
                   double* out, double* tmp0, double* tmp1, cudaStream_t st);
size_t advect_smem_forward(const Geom& g, size_t tsize);
size_t advect_smem_adjoint(const Geom& g, size_t tsize);
bool advect_supported(const Geom& g);

// --- projection and elementwise helpers (poisson_kernels.cu) ---------------
// In-place solenoidal projection of `count` face fields (stride F): Q v = v - G phi
// with (D G) phi = D v.  dct (2D, project_dct_fits): the tables of
// project_dct_tables in T, and phi exactly by the DCT diagonalisation; else an
// on-chip multigrid V(2,2) cycle (vcycles of them).  scratch: (count x
// project_smem / tsize) elements of global memory, required for the multigrid
// when project_needs_scratch (the level arrays then live there, not on chip)
template <class T>
cudaError_t launch_project(const Geom& g, T* fields, int count, int vcycles, cudaStream_t st,
                           T* scratch = nullptr, const T* dct = nullptr);
size_t project_dct_elems(const Geom& g);
bool project_dct_fits(const Geom& g, size_t tsize);
void project_dct_tables(const Geom& g, double* out);
size_t project_smem(const Geom& g, size_t tsize);
bool project_supported(const Geom& g, size_t tsize);
constexpr size_t kProjectSmemLimit = 200 * 1024;   // on-chip layout limit (opt-in 227 KB less static use)
bool project_needs_scratch(const Geom& g, size_t tsize);

template <class T>
void launch_ao_init(const Geom& g, const T* v, const T* lam, double invK, T* w, T* vstar, int warm,
                    cudaStream_t st);
template <class T>
void launch_axpby_faces(const Geom& g, int count, const T* a, double alpha, const T* b, double beta, T* out,
                        cudaStream_t st);
template <class T>
void launch_kkt_force_rhs(const Geom& g, const T* v, T* out, cudaStream_t st);
template <class T>
void launch_kkt_grad_rhs(const Geom& g, const T* v, const T* u, const T* dens, double r, T* out,
                         cudaStream_t st);
template <class T>
void launch_absdiff_max_copy(const T* a, T* b, size_t n, double* out, cudaStream_t st);
// out = x + a (y - x) over count face slabs (the AO blend of Sec. 5)
template <class T>
void launch_blend_faces(const Geom& g, int count, const T* x, const T* y, double a, T* out, cudaStream_t st);
// out += 0.5 * sum_c (rho_c - star_c) * m_c over one cell slab (fp64)
template <class T>
void launch_misfit_dot(const Geom& g, const T* rho, const double* star, const double* m, double* out,
                       cudaStream_t st, RedScratch rs);
// out += scale * sum_e (a_e - b_e)^2 over n entries (fp64)
template <class T>
void launch_diff_sumsq(const T* a, const T* b, size_t n, double scale, double* out, cudaStream_t st,
                       RedScratch rs);

// --- 3D grid (nso3d_kernels.cu, advect3d_kernels.cu, poisson3d_kernels.cu) ---
// Same contracts as the 2D launchers above; the generic launchers forward to
// these when g.dim == 3.
// lamb / lamb_bytes: scratch of the two-pass rows (lamb3_scratch_bytes; NULL:
// the inline form).  Return the kernels launched.
template <class T>
int launch_nso_residual3(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, T sf, T sr,
                         cudaStream_t st, double* sq, const double* only_if_undone, RedScratch rs, void* lamb,
                         size_t lamb_bytes);
template <class T>
int launch_nso_residual3_colour(const Geom& g, CState<T> x, const T* z, CState<T> res, State<T> out, int colour,
                                cudaStream_t st, const double* only_if_undone, void* lamb, size_t lamb_bytes);
// bytes of the two-pass residual scratch of a 3D level (0: the level keeps the inline form)
size_t lamb3_scratch_bytes(const Geom& g, size_t tsize);
size_t lamb3_scratch_bytes_max(const Geom& finest, size_t tsize, const Geom& coarsest, size_t csize);
template <class T>
int launch_scgs3_colour(const Geom& g, State<T> x, CState<T> r, int colour, bool solve_fp32, cudaStream_t st,
                         const double* lm_dev, void* scratch);
size_t scgs3_smem_bytes(int N, size_t tsize);   // shared memory of one cell's SCGS solve
size_t scgs3_thomas_scratch_bytes(const Geom& g, size_t ssize);
template <class Tf, class Tc>
void launch_restrict3(const Geom& gf, const Geom& gc, CState<Tf> s, State<Tc> d, State<Tc> d2, cudaStream_t st);
template <class Tf, class Tc>
void launch_restrict3_faces(const Geom& gf, const Geom& gc, int nt, const Tf* s, Tc* d, cudaStream_t st);
template <class Tf, class Tc>
void launch_prolong3_correct(const Geom& gf, const Geom& gc, State<Tf> f, CState<Tc> cn, CState<Tc> co,
                             cudaStream_t st, const double* undo_if_rose);
template <class T>
void launch_kkt_force_rhs3(const Geom& g, const T* v, T* out, cudaStream_t st);
template <class T>
void launch_kkt_grad_rhs3(const Geom& g, const T* v, const T* u, const T* dens, double r, T* out, cudaStream_t st);
// The 3D sweeps are single cooperative launches over the whole GPU; scratch:
// advect3_scratch_bytes (term buffers and the grid barrier's words).
size_t advect3_scratch_bytes(const Geom& g, size_t tsize);
template <class T>
cudaError_t launch_taylor_forward3(const Geom& g, const T* vel, T* rho, int* K, double thresh, int kmax, int* err,
                                   void* scratch, cudaStream_t st);
template <class T>
cudaError_t launch_taylor_adjoint3(const Geom& g, const T* vel, const T* rho, const int* K, const double* mterm,
                                   T* mu, const T* base, T alpha, T beta, T* out, T* powers, int kmax, int* err,
                                   void* scratch, cudaStream_t st, int s_end = 1, T* mu_m1 = nullptr);
template <class T>
void launch_metric3(const Geom& g, const T* rho_s, const double* star, double c, int levels, double sigma0,
                    double* out, double* tmp0, double* tmp1, cudaStream_t st);
// batched multigrid projection of `count` fields; scratch: project3_scratch_elems(g, count) elements
size_t project3_scratch_elems(const Geom& g, int count);
bool project3_supported(const Geom& g);
template <class T>
cudaError_t launch_project3(const Geom& g, T* fields, int count, int vcycles, cudaStream_t st, T* scratch);
int project3_launches(const Geom& g, int vcycles);

// --- forward simulation and its adjoint (sim_kernels.cu) --------------------
// out = v_prev + dt (u - Adv(v)) (interior faces; walls 0)
template <class T>
void launch_picard_rhs(const Geom& g, const T* v_prev, const T* u, const T* v, double dt, T* out, cudaStream_t st);
// out = y - dt dAdv(v)^T z (interior faces; walls 0)
template <class T>
void launch_picard_adj_rhs(const Geom& g, const T* v, const T* y, const T* z, double dt, T* out, cudaStream_t st);
// out = a x + b y (y may be null)
template <class T>
void launch_sim_axpby(size_t n, double a, const T* x, double b, const T* y, T* out, cudaStream_t st);
// d = scale * s with conversion
template <class Ts, class Td>
void launch_sim_copy(size_t n, const Ts* s, double scale, Td* d, cudaStream_t st);

}  // namespace stc
