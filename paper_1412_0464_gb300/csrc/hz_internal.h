// Internal declarations of the GB300 Helmholtz sweeping solver (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/hz.h"

namespace hz {

// ------------------------------------------------------------------ complex
template <typename R>
struct alignas(2 * sizeof(R)) cplx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { cplx<R> z; z.re = a; z.im = b; return z; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return mk(-a.re, -a.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cconj(cplx<R> a) { return mk(a.re, -a.im); }
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cinv(cplx<R> a) {
  R d = R(1) / (a.re * a.re + a.im * a.im);
  return mk(a.re * d, -a.im * d);
}
template <typename To, typename From>
__host__ __device__ __forceinline__ cplx<To> ccast(cplx<From> a) { return mk((To)a.re, (To)a.im); }

using c64 = cplx<float>;
using c128 = cplx<double>;

// ------------------------------------------------------------------ errors
struct Err {
  hz_status st = HZ_OK;
  std::string msg;
};

#define HZ_CU(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      throw ::hz::Failure(HZ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                  \
  } while (0)

struct Failure {
  hz_status st;
  std::string msg;
  Failure(hz_status s, std::string m) : st(s), msg(std::move(m)) {}
};

// Device error flag codes (written by kernels, read by the host after a call).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADSIZE = 2 };

// ------------------------------------------------------------------ geometry
// One 1-D axis of unknowns: PML factors at the unknowns (node) and at the
// cell midpoints (cell c lies between unknowns c-1 and c), cell sizes.
struct AxisTables {
  int N = 0;                 // unknowns
  c128* a_node = nullptr;    // [N]   alpha at unknowns (device)
  c128* a_cell = nullptr;    // [N+1] alpha at cell midpoints (device)
  double* h_cell = nullptr;  // [N+1] cell sizes (device)
  c64* a_node32 = nullptr;
  c64* a_cell32 = nullptr;
  c128* ia_node = nullptr;   // [N] 1/alpha at unknowns = 1 + i sigma/omega (fine level only)
  c64* ia_node32 = nullptr;
  // unknowns in_lo..in_hi have alpha = 1 exactly at the node and both
  // adjacent cells (the PML-free interior; fine level only, empty if none)
  // and no sponge damping
  int in_lo = 1, in_hi = 0;
  double* beta = nullptr;    // [N] sponge profile at the unknowns (fine level; null: PML)
  float* beta32 = nullptr;
};

// Sponge factor (1 + i beta)^2 of the mass term, beta the sum of the axes'
// profiles (Section 2.1: k -> k (1 + i beta)).
template <typename R>
__host__ __device__ __forceinline__ cplx<R> sponge_s(R beta) {
  return mk<R>((R)1 - beta * beta, (R)2 * beta);
}

// Slab j: core columns lo..hi, wl/wr added PML columns, W = width.
struct Slab {
  int j = 0, lo = 0, hi = 0, wl = 0, wr = 0, W = 0;
  int wp = 0;                // row stride of st, Y, F, E, Phi, Psi: smallest >= W with wp % 8 == 4
  AxisTables ax;             // slab x axis (DD PML in the added columns)
  void* st = nullptr;        // slab stencil [ny][9][wp] in the preconditioner precision
  void* G = nullptr;         // inverse Schur complements [ny][gstride]
  size_t gstride = 0;        // elements per block (W*W rounded up to 16 bytes)
  size_t mstride = 0;        // elements per block of F, E, Phi, Psi (W rows of stride wp)
  void* F = nullptr;         // substitution operators F'_k = G_k L_k [ny][mstride]
  void* E = nullptr;         //   and E'_k = G_k R_k [ny][mstride]
  void* Phi = nullptr;       // forward segment transfer products [P][mstride]
  void* Psi = nullptr;       // backward segment transfer products [P][mstride]
  void* PhiP = nullptr;      // in-group prefix products of Phi [P][mstride] (see Level::grp)
  void* PsiP = nullptr;      // in-group prefix products of Psi [P][mstride]
  void* inj = nullptr;       // injection coefficients [4][ny][3] (T row0, T row1, T~ row0, T~ row1)
  void* Y = nullptr;         // right-hand side, then forward solution rows [ny][n_rhs][wp]
  void* carry_f = nullptr;   // forward segment end values [P+NG][n_rhs][wp] ([P+g]: group g's end)
  void* carry_b = nullptr;   // backward segment start values [P+1+NG][n_rhs][wp] ([P]: meeting
                             // row, [P+1+g]: group g's start)
  // 3-D slabs (dense-block path, slab3d.cu): block rows are the z layers of
  // B = N_y W unknowns (index b = y W + e); G holds [nz][bstride] dense
  // inverses, st3 the slab stencil [nz][27][B] (plane (dz+1) 9 + (dy+1) 3 +
  // (dx+1)), inj3 the transmission coefficients [4][nz][ny][9] ((dz+1) 3 +
  // (dy+1)), Y the forward / solution layers [nz][n_rhs][B], V the two
  // chains' step vectors [2][n_rhs][B].
  int B = 0;
  size_t bstride = 0;
  void* st3 = nullptr;
  void* inj3 = nullptr;
  void* V = nullptr;
  void* gpart = nullptr;     // 3-D: split-K partial sums of the layer GEMM [2][16][max_rhs][B]
  float* Gp = nullptr;       // 3-D complex64, many right-hand sides: G of every layer split
                             //   into TF32 hi / lo planes as tensor-core operand tiles
  float* Vp = nullptr;       //   and the packed right-hand-side blocks of the two chains
  size_t gp_layer = 0;       //   floats per layer of Gp
};

// A grid level on which the sweeping preconditioner (and possibly GMRES) runs.
struct Level {
  bool dim3d = false;        // 3-D level (slabs handled by the dense-block path)
  int nx = 0, ny = 0, nz = 1;  // unknowns along x (sweep), y, z (nz = 1 in 2-D)
  double h = 0;              // uniform spacing (finite differences)
  bool fe = false;           // stored 9-point (2-D) / 27-point (3-D) operator (coarse FE level)
  AxisTables ax, ay, az;
  double* m = nullptr;       // squared slowness at unknowns (FD level), FP64
  float* m32 = nullptr;      // FP32 copy
  c128* st128 = nullptr;     // FE level: 9 / 27 coefficient planes [q][nz][ny][nx]
  c64* st64 = nullptr;
  double* k2c = nullptr;     // FE level: cell k^2 [(nz+1)][(ny+1)][(nx+1)] ((ny+1)(nx+1) in 2-D)
  double* k2ci = nullptr;    // FE level with a sponge: imaginary part of the cell k^2 (else null)
  int* ifp[3] = {};          // FE level, per axis x, y, z: coarse node -> fine node,
  int* refined[3] = {};      //   coarse cell refined flags,
  int* q0[3] = {};           //   prolongation sources per fine node
  int* q1[3] = {};
  size_t size() const { return (size_t)nx * ny * nz; }   // unknowns
  size_t nt() const { return (size_t)ny * nz; }          // transverse unknowns per column
  int planes() const { return dim3d ? 27 : 9; }           // stored stencil planes (FE level)
  int J = 0, w = 0;
  std::vector<int> beta, beta_t;  // Eq. 17, size J+1
  std::vector<Slab> slabs;        // index 1..J (0 unused)
  int mid = 0;                     // meeting row of the two elimination chains
  int P = 2, S0 = 1;               // segments per slab solve; the first S0 on the top chain
  std::vector<int4> seg;           // per segment: first row, rows, direction (+1 / -1), group
  int4* seg_dev = nullptr;
  // Segment groups (two-level carries): consecutive segments of one half;
  // the first G0 groups on the top chain.  Per group: first and last segment,
  // half, index within the half.
  int NG = 2, G0 = 1;
  std::vector<int4> grp;
  int4* grp_dev = nullptr;
  void* fac_desc = nullptr;        // factorisation task descriptors (device, built once)
  int* fac_sync = nullptr;         // their progress / task / group counters (device)
  // 3-D factorisation work (slab3d.cu), allocated by the first factorisation:
  // per chain a dense B x B Schur complement, the panel's colmods [B][NB]
  // and rowmods [NB][B], pivot rows, their inverse map and pivot flags
  void* f3_S = nullptr;
  void* f3_C = nullptr;
  void* f3_R = nullptr;
  int* f3_piv = nullptr;
  float* f3_pack = nullptr;  //   packed tensor-core operands (complex64)
  void* f3_desc = nullptr;
};

// Layout of the parallel-in-y slab substitution for a slab of ny block rows:
// meeting row, segments (first row, rows, direction +1 top / -1 bottom,
// group) and segment groups (first segment, last segment, half, index within
// the half).  segments <= 0: automatic, ~2 ny^(2/3) capped at max_auto.
struct SegmentLayout {
  int mid = 0, P = 0, S0 = 0, G0 = 0, NG = 0;
  std::vector<int4> seg, grp;
};
SegmentLayout segment_layout(int ny, int segments, int max_auto);

// Per-kernel event timing (enabled for roofline reporting): every launch of a
// tagged kernel is bracketed by two events on its own stream.
struct TagTiming {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t used = 0;
  double ms = 0;
  long long launches = 0;
  double bytes = 0;
};
struct Timing {
  bool on = false;
  std::map<std::string, TagTiming> tags;   // node-based: references stay valid
  TagTiming& tag(const std::string& name) { return tags[name]; }
};
// Records start/stop events around `launch` when timing is on.
template <typename F>
void timed(hz_handle* h, const char* tag, double bytes, cudaStream_t s, F&& launch);

}  // namespace hz

struct hz_handle {
  hz_params p{};
  hz::Err err;
  int dev = 0;
  int sms = 1;               // multiprocessors of the device
  double c_pml = 0;
  hz::Level fine;            // the PDE grid (GMRES level)
  hz::Level coarse;          // two-grid coarse level (sweeps), if p.two_grid
  hz::Level* sweep = nullptr;  // level carrying the DD (fine or coarse)
  bool factored = false;
  int* dev_flag = nullptr;   // device error flag
  // preconditioner work (precision of the preconditioner), per level
  void* pr_r = nullptr;      // input residual on the sweep level [max_rhs][n]
  void* pr_u = nullptr;      // output on the sweep level
  void* pr_u2 = nullptr;     // second sweep phase output on the sweep level
  void* pr_g = nullptr;      // mid-sweep residual g = f - A u
  void* pr_B1 = nullptr;     // transmission buffers [2][max_rhs][N_t]
  void* pr_B2 = nullptr;
  void* pr_Bnx = nullptr;    // NX-sweep: 2 n_cell + 2 transmission buffers [2][max_rhs][N_t]
  void* tg_u = nullptr;      // two-grid fine work (preconditioner precision)
  void* tg_r = nullptr;
  void* tg_t = nullptr;
  // GMRES (FP64)
  hz::c128* V = nullptr;     // [(m+1)][max_rhs][n]
  hz::c128* Z = nullptr;     // [m][max_rhs][n]
  hz::c128* W = nullptr;     // [max_rhs][n] work
  hz::c128* R = nullptr;     // [max_rhs][n] residual
  double* red = nullptr;     // reduction scratch
  hz::c128* hcol = nullptr;  // [max_rhs][m+1] Hessenberg column on device
  cudaStream_t s2 = nullptr; // second stream for the concurrent chain of the X-sweep
  cudaEvent_t evA = nullptr, evB = nullptr;
  hz::Timing timing;
  hz_stats stats{};
  long long launches = 0;
  hz::c128* stage_f = nullptr;  // host-call staging buffers [max_rhs][n]
  hz::c128* stage_u = nullptr;
  hz::c128* gr_b = nullptr;     // gradient work [max_rhs][n]: right-hand sides,
  hz::c128* gr_u = nullptr;     //   forward fields,
  hz::c128* gr_mu = nullptr;    //   adjoint fields
  double* gr_phi = nullptr;     //   per right-hand-side misfit [max_rhs]
  void* gm_state = nullptr;     // GMRES Arnoldi state (Hessenberg, rotations, ...) [max_rhs]
  // CUDA graphs of the preconditioner application inside GMRES, one per
  // (input, output, n_rhs); valid while the levels' buffers stay allocated
  struct PrecGraph {
    const void* in;
    void* out;
    int nr;
    cudaGraphExec_t exec;
    long long launches;         // kernels in the graph
  };
  std::vector<PrecGraph> pgraphs;
  std::vector<int> pwarm;       // n_rhs values whose preconditioner has run once uncaptured
};

namespace hz {
template <typename F>
void timed(hz_handle* h, const char* tag, double bytes, cudaStream_t s, F&& launch) {
  if (!h->timing.on) {
    launch();
    return;
  }
  TagTiming& t = h->timing.tag(tag);
  if (t.used == t.ev.size()) {
    cudaEvent_t a, b;
    HZ_CU(cudaEventCreate(&a));
    HZ_CU(cudaEventCreate(&b));
    t.ev.push_back({a, b});
  }
  auto& e = t.ev[t.used++];
  HZ_CU(cudaEventRecord(e.first, s));
  launch();
  HZ_CU(cudaEventRecord(e.second, s));
  t.launches++;
  t.bytes += bytes;
}
}  // namespace hz

namespace hz {

// setup.cu
void build_level_fd(hz_handle* h, Level& L, const int* n_int, int w_out, double hh,
                    const double* m_dev, bool dim3d, cudaStream_t s);
void build_level_fe(hz_handle* h, Level& L, const Level& fine, const int* n_int, int w_out,
                    double hh, cudaStream_t s);
void build_slabs(hz_handle* h, Level& L, cudaStream_t s);
void partition(Level& L);
void slab_geometry(hz_handle* h, Level& L, Slab& S, int j, cudaStream_t s);
void free_level(Level& L);
double mean_velocity(const double* m_dev, size_t n, cudaStream_t s);

// stencil.cu: fine 5-point operator (on the fly) or stored 9-point operator.
template <typename R>
void level_residual(hz_handle* h, const Level& L, const cplx<R>* f, const cplx<R>* u,
                    cplx<R>* r, int n_rhs, cudaStream_t s);  // r = f - A u (f may be null: r = -A u)
template <typename R>
void level_apply(hz_handle* h, const Level& L, const cplx<R>* u, cplx<R>* y, int n_rhs,
                 cudaStream_t s);
template <typename R>
void jacobi_steps(hz_handle* h, const Level& L, const cplx<R>* f, cplx<R>* u, cplx<R>* t,
                  int nu, double omega_jac, int n_rhs, cudaStream_t s);
template <typename R>
void restrict_residual(hz_handle* h, const Level& F, const Level& C, const cplx<R>* rf,
                       cplx<R>* rc, int n_rhs, cudaStream_t s);
template <typename R>
void prolong_add(hz_handle* h, const Level& F, const Level& C, const cplx<R>* ec, cplx<R>* uf,
                 int n_rhs, cudaStream_t s);

template <typename R>
void slab_stencil_fe(hz_handle* h, const Level& L, const Slab& S, cudaStream_t s);

// slab.cu
template <typename R>
void factor_level(hz_handle* h, Level& L, cudaStream_t s);
struct SolveSpec;  // defined in slab.cu
template <typename R>
void subdom_solve(hz_handle* h, Level& L, int j, const cplx<R>* f, int a, int b, int at, int bt,
                  bool tau1, const cplx<R>* B1, bool tau2, cplx<R>* B2, bool tau3,
                  const cplx<R>* B3, bool tau4, cplx<R>* B4, cplx<R>* u, int n_rhs,
                  cudaStream_t s);
template <typename R>
void slab_solve_raw(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud, int n_rhs,
                    cudaStream_t s);
template <typename R>
void slab_solve_raw_scratch(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud,
                            int n_rhs, cudaStream_t s, cplx<R>* Y, cplx<R>* carry_f,
                            cplx<R>* carry_b);

// slab3d.cu: 3-D slabs (block rows = z layers, dense B x B blocks)
template <typename R>
void build_slabs3d(hz_handle* h, Level& L, cudaStream_t s);
template <typename R>
void factor_level3d(hz_handle* h, Level& L, cudaStream_t s);
template <typename R>
void subdom_solve3d(hz_handle* h, Level& L, int j, const cplx<R>* f, int a, int b, int at,
                    int bt, bool tau1, const cplx<R>* B1, bool tau2, cplx<R>* B2, bool tau3,
                    const cplx<R>* B3, bool tau4, cplx<R>* B4, cplx<R>* u, int n_rhs,
                    cudaStream_t s);
template <typename R>
void slab_solve_raw3d(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud, int n_rhs,
                      cudaStream_t s);

// stencil3d.cu: 3-D operators (fine 7-point on the fly, coarse 27-point stored)
template <typename R>
void launch_op3d(hz_handle* h, const Level& L, int mode, const cplx<R>* f, const cplx<R>* u,
                 cplx<R>* y, int n_rhs, double omega_jac, cudaStream_t s);

// sweep.cu
template <typename R>
void sweep_apply(hz_handle* h, Level& L, const cplx<R>* f, cplx<R>* u, int n_rhs,
                 cudaStream_t s);  // u = P f (P_X or P_UD)
void precond_apply(hz_handle* h, const c128* r, c128* z, int n_rhs, cudaStream_t s);
// The same through a captured CUDA graph (GMRES); clear_graphs drops them.
void precond_graphed(hz_handle* h, const c128* r, c128* z, int n_rhs, cudaStream_t s);
void clear_graphs(hz_handle* h);

// gmres.cu
void gmres_solve(hz_handle* h, const c128* f, c128* u, int n_rhs, cudaStream_t s);
void misfit_grad(hz_handle* h, const int* src, int n_src, const int* rec, int n_rec,
                 const c128* d, double* grad, double* phi_out, cudaStream_t s);
void apply_fine64(hz_handle* h, const c128* u, c128* y, int n_rhs, cudaStream_t s);

// api.cu: runs `body`, maps hz::Failure, std::exception and a pending CUDA
// error to a status (recorded in the handle), never throws.
hz_status run_guarded(hz_handle* h, const std::function<void()>& body);

// util
template <typename To, typename From>
void cast_copy(const cplx<From>* a, cplx<To>* b, size_t n, cudaStream_t s);
void check_dev_flag(hz_handle* h, cudaStream_t s);
inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
void* dmalloc(size_t bytes);
void dfree(void* p);
// Test hook: the integer value of environment variable `name`, or -1 if it
// is unset or not a number (read at every call; see include/hz.h).
long long test_hook(const char* name);

}  // namespace hz
