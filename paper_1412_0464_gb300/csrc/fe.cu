// Coarse level of the two-grid sweeping preconditioner (Section 4, Appendix A).
//
// * PML-aware coarsening (Section 4.2): per axis the w_out PML cells are kept
//   and the n interior cells are merged in pairs; coarse node Q sits at fine
//   node i_FP(Q); r_C(Q + 1/2) tells whether coarse cell Q + 1/2 is refined.
// * Coarse cell k^2 (Appendix A.3, last paragraph): tensor averaging of the
//   fine nodal k^2 with weights (1/2, 1/2) across an unrefined cell and
//   (1/4, 1/2, 1/4) across a refined one.
// * Optimised FE operator (Appendix A.2-A.3, Eqs. 54-63, Table 9): per cell
//   the constants I_a, J_b from c_j(1/G), G = 2 pi / (H k_cell), linearly
//   interpolated in Table 9 (2-D: I0 = c1/4, I1 = c2/8, I2 = (1-c1-c2)/4,
//   J0 = c3/2, J1 = (1-c3)/2).  A cell with corners a, b contributes
//     -vol I_{|a-b|} k^2/(alpha_x alpha_y)
//     - sum_l sgn_l (alpha_l / h_l)(h_m / alpha_m) J_{|a_m - b_m|},
//   sgn_l = -1 if a_l == b_l else +1, to the entry (node a, node b).
// * Transfer (Eqs. 41-42): P by tent functions on the coarse mesh, R = P^T.
#include "hz_internal.h"

#include <cmath>

namespace hz {

// Table 9 (a): 1/G_k = 0, 0.04, ..., 0.40 and c1, c2, c3 (2-D).
__constant__ double kTable9_2d[11][3] = {
    {0.61953, 0.45295, 0.77363}, {0.63691, 0.47535, 0.87242}, {0.62988, 0.48633, 0.86400},
    {0.62610, 0.48880, 0.84984}, {0.62289, 0.48759, 0.83017}, {0.62596, 0.47106, 0.80852},
    {0.62213, 0.46478, 0.78215}, {0.61036, 0.47016, 0.74857}, {0.59107, 0.48468, 0.70553},
    {0.56369, 0.50746, 0.65062}, {0.52412, 0.54163, 0.57676}};

__device__ __forceinline__ c128 pml_alpha_fe(double sigma, double omega) {
  double a = sigma / omega;
  double d = 1.0 / (1.0 + a * a);
  return mk(d, -a * d);
}

__device__ __forceinline__ int coarse_to_fine(int Q, int w_out, int n_int) {
  const int half = n_int / 2;
  if (Q <= w_out) return Q;
  if (Q <= w_out + half) return w_out + 2 * (Q - w_out);
  return Q + half;
}

// Coarse axis: cell sizes and alpha at coarse cell midpoints / unknowns, plus
// the fine-node map i_FP and the refinement flags.
__global__ void coarse_axis_kernel(int n_c, int w_out, int n_int, double h, double C, double omega,
                                   c128* a_node, c128* a_cell, double* h_cell, c64* a_node32,
                                   c64* a_cell32, int* ifp, int* refined) {
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  if (Q > n_c) return;
  const double lo = w_out * h, hi = (2 * w_out + n_int - w_out) * h;
  auto sigma = [&](double x) {
    double d = fmax(0.0, fmax(lo - x, x - hi));
    return C * d * d;
  };
  const int p = coarse_to_fine(Q, w_out, n_int);
  ifp[Q] = p;
  if (Q < n_c) {
    const int p1 = coarse_to_fine(Q + 1, w_out, n_int);
    refined[Q] = (p1 - p == 2);
    const double xm = 0.5 * (p + p1) * h;
    const c128 a = pml_alpha_fe(sigma(xm), omega);
    a_cell[Q] = a;
    a_cell32[Q] = ccast<float>(a);
    h_cell[Q] = (p1 - p) * h;
  }
  if (Q >= 1 && Q < n_c) {
    const c128 a = pml_alpha_fe(sigma(p * h), omega);
    a_node[Q - 1] = a;
    a_node32[Q - 1] = ccast<float>(a);
  }
}

// Coarse cell k^2 = omega^2 * average of the fine nodal m (edge values at the
// Dirichlet nodes), tensor product of the 1-D weights.
__global__ void coarse_k2_kernel(int n_c, int N_fine, const int* ifp, const int* refined,
                                 const double* m_fine, double omega2, double* k2c) {
  const int cx = blockIdx.x * blockDim.x + threadIdx.x;
  const int cy = blockIdx.y;
  if (cx >= n_c || cy >= n_c) return;
  double wy[3], wx[3];
  const int ry = refined[cy], rx = refined[cx];
  const int py = ifp[cy], px = ifp[cx];
  if (ry) { wy[0] = 0.25; wy[1] = 0.5; wy[2] = 0.25; } else { wy[0] = 0.5; wy[1] = 0.5; wy[2] = 0.0; }
  if (rx) { wx[0] = 0.25; wx[1] = 0.5; wx[2] = 0.25; } else { wx[0] = 0.5; wx[1] = 0.5; wx[2] = 0.0; }
  double acc = 0;
  for (int a = 0; a < 3; ++a) {
    if (wy[a] == 0.0) continue;
    const int uy = min(max(py + a - 1, 0), N_fine - 1);   // fine node -> unknown, edge-padded
    for (int b = 0; b < 3; ++b) {
      if (wx[b] == 0.0) continue;
      const int ux = min(max(px + b - 1, 0), N_fine - 1);
      acc += wy[a] * wx[b] * m_fine[(size_t)uy * N_fine + ux];
    }
  }
  k2c[(size_t)cy * n_c + cx] = omega2 * acc;
}

__device__ __forceinline__ void table9_2d(double inv_G, double c[3]) {
  double x = fmin(fmax(inv_G, 0.0), 0.40);
  int idx = (int)floor(x / 0.04);
  if (idx > 9) idx = 9;
  if (idx < 0) idx = 0;
  const double t = (x - 0.04 * idx) / 0.04;
  for (int q = 0; q < 3; ++q) c[q] = (1.0 - t) * kTable9_2d[idx][q] + t * kTable9_2d[idx + 1][q];
}

struct FeMesh {
  int nx, ny;                 // unknowns of the output mesh
  const double* hx;           // [nx+1]
  const c128* ax;             // [nx+1]
  const double* hy;           // [ny+1]
  const c128* ay;             // [ny+1]
  const double* k2c;          // global cell k^2, [ny+1][k2_ld]
  int k2_ld;
  int lo, hi, wl;             // column of cell cx in k2c: clamp(cx - wl + lo, lo, hi + 1)
  double H, omega;            // reference spacing for G
  size_t sq, sk, sx;          // output index = q*sq + k*sk + x*sx, q = (dy+1)*3 + (dx+1)
};

// Assemble the 9-point FE stencil of every unknown of the mesh.
template <typename R>
__global__ void fe_assemble_kernel(FeMesh ms, cplx<R>* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (x >= ms.nx || k >= ms.ny) return;
  c128 acc[9];
  for (int q = 0; q < 9; ++q) acc[q] = mk(0.0, 0.0);
  for (int cyo = 0; cyo < 2; ++cyo) {
    const int cy = k + cyo;                  // cells k (below) and k+1 (above)
    const int ay_ = cyo == 0 ? 1 : 0;        // node's corner index in the cell along y
    for (int cxo = 0; cxo < 2; ++cxo) {
      const int cx = x + cxo;
      const int ax_ = cxo == 0 ? 1 : 0;
      const int gcx = min(max(cx - ms.wl + ms.lo, ms.lo), ms.hi + 1);
      const double k2 = ms.k2c[(size_t)cy * ms.k2_ld + gcx];
      const double hx = ms.hx[cx], hy = ms.hy[cy];
      const c128 alx = ms.ax[cx], aly = ms.ay[cy];
      double c[3];
      table9_2d(ms.H * sqrt(k2) / (2.0 * M_PI), c);
      const double I[3] = {c[0] / 4, c[1] / 8, (1 - c[0] - c[1]) / 4};
      const double Jc[2] = {c[2] / 2, (1 - c[2]) / 2};
      const c128 mass = (hx * hy * k2) * cinv(alx * aly);
      const c128 sx_ = (hy / hx) * (alx * cinv(aly));    // (alpha_x/h_x)(h_y/alpha_y)
      const c128 sy_ = (hx / hy) * (aly * cinv(alx));    // (alpha_y/h_y)(h_x/alpha_x)
      for (int by = 0; by < 2; ++by) {
        const int ny_ = cy + by - 1;           // neighbour unknown along y
        if (ny_ < 0 || ny_ >= ms.ny) continue;
        for (int bx = 0; bx < 2; ++bx) {
          const int nx_ = cx + bx - 1;
          if (nx_ < 0 || nx_ >= ms.nx) continue;
          const int ham = (ay_ != by) + (ax_ != bx);
          c128 v = -(I[ham] * mass);
          const double sgx = (ax_ == bx) ? -1.0 : 1.0;
          const double sgy = (ay_ == by) ? -1.0 : 1.0;
          v = v - (sgx * Jc[ay_ != by]) * sx_;
          v = v - (sgy * Jc[ax_ != bx]) * sy_;
          const int q = (ny_ - k + 1) * 3 + (nx_ - x + 1);
          acc[q] = acc[q] + v;
        }
      }
    }
  }
  for (int q = 0; q < 9; ++q)
    out[q * ms.sq + (size_t)k * ms.sk + (size_t)x * ms.sx] = ccast<R>(acc[q]);
}

// r_c = P^T r_f (Section 4.2: R is the transpose of the prolongation).
template <typename R>
__global__ void restrict_kernel(int n_c, int N_f, const int* ifp, const int* refined,
                                const cplx<R>* rf, cplx<R>* rc, int nr) {
  const int qx = blockIdx.x * blockDim.x + threadIdx.x;   // coarse unknown, node qx + 1
  const int qy = blockIdx.y;
  const int r = blockIdx.z;
  const int Nc = n_c - 1;
  if (qx >= Nc || qy >= Nc) return;
  const int Qx = qx + 1, Qy = qy + 1;
  double wy[3] = {refined[Qy - 1] ? 0.5 : 0.0, 1.0, refined[Qy] ? 0.5 : 0.0};
  double wx[3] = {refined[Qx - 1] ? 0.5 : 0.0, 1.0, refined[Qx] ? 0.5 : 0.0};
  const int py = ifp[Qy], px = ifp[Qx];
  cplx<R> acc = mk<R>(0, 0);
  const cplx<R>* f = rf + (size_t)r * N_f * N_f;
  for (int a = 0; a < 3; ++a) {
    if (wy[a] == 0.0) continue;
    const int uy = py + a - 2;               // fine node (py + a - 1) -> unknown
    for (int b = 0; b < 3; ++b) {
      if (wx[b] == 0.0) continue;
      const int ux = px + b - 2;
      const cplx<R> v = f[(size_t)uy * N_f + ux];
      acc = acc + (R)(wy[a] * wx[b]) * v;
    }
  }
  rc[(size_t)r * Nc * Nc + (size_t)qy * Nc + qx] = acc;
}

// Per fine node (1..n_f_cells-1): coarse sources of the prolongation:
// node i_FP(Q) takes e_Q; node i_FP(Q)+1 in a refined cell takes (e_Q + e_{Q+1})/2.
__global__ void prolong_map_kernel(int n_c, const int* ifp, const int* refined, int* q0, int* q1) {
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  if (Q > n_c) return;
  const int p = ifp[Q];
  q0[p] = Q;
  q1[p] = -1;
  if (Q < n_c && refined[Q]) {
    q0[p + 1] = Q;
    q1[p + 1] = Q + 1;
  }
}

// u_f += P e_c
template <typename R>
__global__ void prolong_add_kernel(int N_f, int n_c, const int* q0, const int* q1,
                                   const cplx<R>* ec, cplx<R>* uf, int nr) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;   // fine unknown, node x + 1
  const int y = blockIdx.y;
  const int r = blockIdx.z;
  if (x >= N_f || y >= N_f) return;
  const int Nc = n_c - 1;
  const cplx<R>* e = ec + (size_t)r * Nc * Nc;
  auto val = [&](int Qy, int Qx) -> cplx<R> {   // Dirichlet coarse nodes carry zero
    if (Qy <= 0 || Qy >= n_c || Qx <= 0 || Qx >= n_c) return mk<R>(0, 0);
    return e[(size_t)(Qy - 1) * Nc + (Qx - 1)];
  };
  const int ay0 = q0[y + 1], ay1 = q1[y + 1], ax0 = q0[x + 1], ax1 = q1[x + 1];
  const R wy = ay1 >= 0 ? (R)0.5 : (R)1, wx = ax1 >= 0 ? (R)0.5 : (R)1;
  cplx<R> v = (wy * wx) * val(ay0, ax0);
  if (ax1 >= 0) v = v + (wy * wx) * val(ay0, ax1);
  if (ay1 >= 0) {
    v = v + (wy * wx) * val(ay1, ax0);
    if (ax1 >= 0) v = v + (wy * wx) * val(ay1, ax1);
  }
  cplx<R>* u = uf + (size_t)r * N_f * N_f + (size_t)y * N_f + x;
  *u = *u + v;
}

// ---------------------------------------------------------------- host side
static void alloc_axis_fe(AxisTables& a, int N) {
  a.N = N;
  a.a_node = (c128*)dmalloc(sizeof(c128) * N);
  a.a_cell = (c128*)dmalloc(sizeof(c128) * (N + 1));
  a.h_cell = (double*)dmalloc(sizeof(double) * (N + 1));
  a.a_node32 = (c64*)dmalloc(sizeof(c64) * N);
  a.a_cell32 = (c64*)dmalloc(sizeof(c64) * (N + 1));
}

void build_level_fe(hz_handle* h, Level& L, const Level& fine, int n, int w_out, double hh,
                    cudaStream_t s) {
  const int n_c = 2 * w_out + n / 2;      // coarse cells per axis
  L.nx = L.ny = n_c - 1;
  L.h = 2 * hh;                            // interior coarse spacing H
  L.fe = true;
  const double C = (w_out > 0) ? h->p.s_pml_out * h->c_pml / std::pow(w_out * hh, 3) : 0.0;
  L.ifp = (int*)dmalloc(sizeof(int) * (n_c + 1));
  L.refined = (int*)dmalloc(sizeof(int) * (n_c + 1));
  for (AxisTables* a : {&L.ax, &L.ay}) {
    alloc_axis_fe(*a, L.nx);
    coarse_axis_kernel<<<cdiv(n_c + 1, 128), 128, 0, s>>>(n_c, w_out, n, hh, C, h->p.omega,
                                                          a->a_node, a->a_cell, a->h_cell,
                                                          a->a_node32, a->a_cell32, L.ifp,
                                                          L.refined);
  }
  L.k2c = (double*)dmalloc(sizeof(double) * (size_t)n_c * n_c);
  coarse_k2_kernel<<<dim3(cdiv(n_c, 128), n_c), 128, 0, s>>>(n_c, fine.nx, L.ifp, L.refined,
                                                              fine.m, h->p.omega * h->p.omega, L.k2c);
  const size_t plane = (size_t)L.nx * L.ny;
  L.st128 = (c128*)dmalloc(sizeof(c128) * 9 * plane);
  L.st64 = (c64*)dmalloc(sizeof(c64) * 9 * plane);
  FeMesh ms{L.nx, L.ny, L.ax.h_cell, L.ax.a_cell, L.ay.h_cell, L.ay.a_cell, L.k2c, n_c,
            0, L.nx - 1, 0, L.h, h->p.omega, plane, (size_t)L.nx, 1};
  dim3 grid(cdiv(L.nx, 128), L.ny);
  fe_assemble_kernel<double><<<grid, 128, 0, s>>>(ms, L.st128);
  fe_assemble_kernel<float><<<grid, 128, 0, s>>>(ms, L.st64);
  // prolongation maps (fine node -> coarse sources)
  const int nf_cells = 2 * w_out + n;
  L.q0 = (int*)dmalloc(sizeof(int) * (nf_cells + 1));
  L.q1 = (int*)dmalloc(sizeof(int) * (nf_cells + 1));
  prolong_map_kernel<<<cdiv(n_c + 1, 128), 128, 0, s>>>(n_c, L.ifp, L.refined, L.q0, L.q1);
  HZ_CU(cudaGetLastError());
  HZ_CU(cudaStreamSynchronize(s));
}

// Slab stencil of the coarse FE operator on the extended slab mesh: cell k^2
// frozen to the interface cell in the added PML (Eq. 10, cellwise).
template <typename R>
void slab_stencil_fe(hz_handle* h, const Level& L, const Slab& S, cudaStream_t s) {
  FeMesh ms{S.W, L.ny, S.ax.h_cell, S.ax.a_cell, L.ay.h_cell, L.ay.a_cell, L.k2c, L.nx + 1,
            S.lo, S.hi, S.wl, L.h, h->p.omega, (size_t)S.wp, (size_t)9 * S.wp, 1};
  dim3 grid(cdiv(S.W, 128), L.ny);
  fe_assemble_kernel<R><<<grid, 128, 0, s>>>(ms, (cplx<R>*)S.st);
  HZ_CU(cudaGetLastError());
}

template <typename R>
void restrict_residual(hz_handle* h, const Level& F, const Level& C, const cplx<R>* rf,
                       cplx<R>* rc, int n_rhs, cudaStream_t s) {
  dim3 grid(cdiv(C.nx, 128), C.ny, n_rhs);
  restrict_kernel<R><<<grid, 128, 0, s>>>(C.nx + 1, F.nx, C.ifp, C.refined, rf, rc, n_rhs);
  h->launches++;
  HZ_CU(cudaGetLastError());
}

template <typename R>
void prolong_add(hz_handle* h, const Level& F, const Level& C, const cplx<R>* ec, cplx<R>* uf,
                 int n_rhs, cudaStream_t s) {
  dim3 grid(cdiv(F.nx, 128), F.ny, n_rhs);
  prolong_add_kernel<R><<<grid, 128, 0, s>>>(F.nx, C.nx + 1, C.q0, C.q1, ec, uf, n_rhs);
  h->launches++;
  HZ_CU(cudaGetLastError());
}

template void slab_stencil_fe<float>(hz_handle*, const Level&, const Slab&, cudaStream_t);
template void slab_stencil_fe<double>(hz_handle*, const Level&, const Slab&, cudaStream_t);
template void restrict_residual<float>(hz_handle*, const Level&, const Level&, const c64*, c64*, int,
                                       cudaStream_t);
template void restrict_residual<double>(hz_handle*, const Level&, const Level&, const c128*, c128*,
                                        int, cudaStream_t);
template void prolong_add<float>(hz_handle*, const Level&, const Level&, const c64*, c64*, int,
                                 cudaStream_t);
template void prolong_add<double>(hz_handle*, const Level&, const Level&, const c128*, c128*, int,
                                  cudaStream_t);

}  // namespace hz
