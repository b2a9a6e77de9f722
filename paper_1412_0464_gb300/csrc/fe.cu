// Coarse level of the two-grid sweeping preconditioner (Section 4, Appendix A).
//
// * PML-aware coarsening (Section 4.2): per axis the w_out PML cells are kept
//   and the n interior cells are merged in pairs; coarse node Q sits at fine
//   node i_FP(Q); r_C(Q + 1/2) tells whether coarse cell Q + 1/2 is refined.
//   Every axis has its own cell count (rectangles and boxes).
// * Coarse cell k^2 (Appendix A.3, last paragraph): tensor averaging of the
//   fine nodal k^2 with weights (1/2, 1/2) across an unrefined cell and
//   (1/4, 1/2, 1/4) across a refined one.
// * Optimised FE operator (Appendix A.2-A.3, Eqs. 54-63, Table 9): per cell
//   the constants I_a, J_b from c_j(1/G), G = 2 pi / (H k_cell), linearly
//   interpolated in Table 9 (2-D: I0 = c1/4, I1 = c2/8, I2 = (1-c1-c2)/4,
//   J0 = c3/2, J1 = (1-c3)/2; 3-D, Eq. 63: I0 = c1/8, I1 = c2/24,
//   I2 = c3/24, I3 = (1-c1-c2-c3)/8, J0 = c4/4, J1 = c5/8, J2 = (1-c4-c5)/4).
//   A cell with corners a, b contributes
//     -vol I_{|a-b|} k^2 / prod_l alpha_l
//     - sum_l sgn_l (alpha_l / h_l) prod_{m != l} (h_m / alpha_m) J_{|a-b| off axis l},
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

// Table 9 (b): 1/G_k = 0, 0.04, ..., 0.40 and c1 .. c5 (3-D).
__constant__ double kTable9_3d[11][5] = {
    {0.56428, 0.35970, 0.20490, 0.77998, 0.17505}, {0.56571, 0.36071, 0.20541, 0.78635, 0.17442},
    {0.56298, 0.36150, 0.20719, 0.78273, 0.16881}, {0.56540, 0.35620, 0.20287, 0.76438, 0.18678},
    {0.56370, 0.35299, 0.20299, 0.74684, 0.19603}, {0.55813, 0.35277, 0.20452, 0.72755, 0.20131},
    {0.54673, 0.35830, 0.20693, 0.70298, 0.20847}, {0.52423, 0.38368, 0.19633, 0.66863, 0.22424},
    {0.49946, 0.39740, 0.20725, 0.62734, 0.23845}, {0.47567, 0.40216, 0.22132, 0.58198, 0.25329},
    {0.45011, 0.36784, 0.29962, 0.53417, 0.23589}};

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
  } else {
    refined[Q] = 0;
  }
  if (Q >= 1 && Q < n_c) {
    const c128 a = pml_alpha_fe(sigma(p * h), omega);
    a_node[Q - 1] = a;
    a_node32[Q - 1] = ccast<float>(a);
  }
}

// One axis of the coarse k^2 averaging: the (up to) three fine unknowns
// (edge-padded: the Dirichlet nodes take the edge values) and their weights.
struct Avg1 {
  int u[3];
  double w[3];
};
__device__ __forceinline__ Avg1 avg_axis(int c, const int* ifp, const int* refined, int N_fine) {
  Avg1 a;
  const int p = ifp[c];
  const bool r = refined[c] != 0;
  a.w[0] = r ? 0.25 : 0.5;
  a.w[1] = r ? 0.5 : 0.5;
  a.w[2] = r ? 0.25 : 0.0;
  for (int t = 0; t < 3; ++t) a.u[t] = min(max(p + t - 1, 0), N_fine - 1);   // fine node -> unknown
  return a;
}

// Coarse cell k^2 = omega^2 * tensor average of the fine nodal m (times the
// sponge factor (1 + i beta)^2 when the fine level has a sponge: k2ci then
// receives the imaginary part).  2-D: z axis trivial (ncz = 1, the single
// weight 1).
__global__ void coarse_k2_kernel(int ncx, int ncy, int ncz, int Nfx, int Nfy, int Nfz,
                                 const int* ifpx, const int* refx, const int* ifpy,
                                 const int* refy, const int* ifpz, const int* refz,
                                 const double* m_fine, double omega2, double* k2c,
                                 const double* bfx, const double* bfy, const double* bfz,
                                 double* k2ci) {
  const int cx = blockIdx.x * blockDim.x + threadIdx.x;
  const int cy = blockIdx.y, cz = blockIdx.z;
  if (cx >= ncx || cy >= ncy || cz >= ncz) return;
  const Avg1 ax = avg_axis(cx, ifpx, refx, Nfx), ay = avg_axis(cy, ifpy, refy, Nfy);
  Avg1 az;
  if (ifpz) {
    az = avg_axis(cz, ifpz, refz, Nfz);
  } else {
    az.u[0] = az.u[1] = az.u[2] = 0;
    az.w[0] = 0.0; az.w[1] = 1.0; az.w[2] = 0.0;
  }
  c128 acc = mk(0.0, 0.0);
  for (int c = 0; c < 3; ++c) {
    if (az.w[c] == 0.0) continue;
    for (int a = 0; a < 3; ++a) {
      if (ay.w[a] == 0.0) continue;
      for (int b = 0; b < 3; ++b) {
        if (ax.w[b] == 0.0) continue;
        const double wm = az.w[c] * ay.w[a] * ax.w[b] *
                          m_fine[((size_t)az.u[c] * Nfy + ay.u[a]) * Nfx + ax.u[b]];
        if (bfx) {
          const double beta = bfx[ax.u[b]] + bfy[ay.u[a]] + (bfz ? bfz[az.u[c]] : 0.0);
          acc = acc + wm * sponge_s(beta);
        } else {
          acc.re += wm;
        }
      }
    }
  }
  const size_t o = ((size_t)cz * ncy + cy) * ncx + cx;
  k2c[o] = omega2 * acc.re;
  if (k2ci) k2ci[o] = omega2 * acc.im;
}

// The cell's complex k^2 and the real wavenumber Re sqrt(k^2) used for G
// (in a sponge k^2 (1 + i beta)^2 -> k; the damping does not change the
// Table 9 coefficients).
__device__ __forceinline__ c128 cell_k2(const double* k2c, const double* k2ci, size_t o,
                                        double* kreal) {
  const double re = k2c[o], im = k2ci ? k2ci[o] : 0.0;
  const double mod = sqrt(re * re + im * im);
  *kreal = sqrt(fmax(0.0, 0.5 * (mod + re)));
  return mk(re, im);
}

__device__ __forceinline__ void table9_2d(double inv_G, double c[3]) {
  double x = fmin(fmax(inv_G, 0.0), 0.40);
  int idx = (int)floor(x / 0.04);
  if (idx > 9) idx = 9;
  if (idx < 0) idx = 0;
  const double t = (x - 0.04 * idx) / 0.04;
  for (int q = 0; q < 3; ++q) c[q] = (1.0 - t) * kTable9_2d[idx][q] + t * kTable9_2d[idx + 1][q];
}

__device__ __forceinline__ void table9_3d(double inv_G, double c[5]) {
  double x = fmin(fmax(inv_G, 0.0), 0.40);
  int idx = (int)floor(x / 0.04);
  if (idx > 9) idx = 9;
  if (idx < 0) idx = 0;
  const double t = (x - 0.04 * idx) / 0.04;
  for (int q = 0; q < 5; ++q) c[q] = (1.0 - t) * kTable9_3d[idx][q] + t * kTable9_3d[idx + 1][q];
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
  const double* k2ci;         // imaginary part of the cell k^2 (sponge) or null
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
      double kr;
      const c128 k2 = cell_k2(ms.k2c, ms.k2ci, (size_t)cy * ms.k2_ld + gcx, &kr);
      const double hx = ms.hx[cx], hy = ms.hy[cy];
      const c128 alx = ms.ax[cx], aly = ms.ay[cy];
      double c[3];
      table9_2d(ms.H * kr / (2.0 * M_PI), c);
      const double I[3] = {c[0] / 4, c[1] / 8, (1 - c[0] - c[1]) / 4};
      const double Jc[2] = {c[2] / 2, (1 - c[2]) / 2};
      const c128 mass = (hx * hy) * (k2 * cinv(alx * aly));
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

// 3-D mesh of the 27-point FE stencil: per axis cell sizes and alpha at cell
// midpoints (cells 0..N along each axis), the global cell k^2
// [(nz+1)][(ny+1)][k2_ld] with the x cell column clamp of a slab, and the
// output strides (index q*sq + z*sz + y*sy + x*sx, q = (dz+1) 9 + (dy+1) 3 + (dx+1)).
struct FeMesh3 {
  int nx, ny, nz;
  const double* h[3];         // x, y, z cell sizes
  const c128* a[3];           // x, y, z alpha at cell midpoints
  const double* k2c;
  int k2_ld, k2_ny1;          // k2c row length (x cells) and rows per plane (ny + 1)
  int lo, hi, wl;
  double H, omega;
  size_t sq, sz, sy, sx;
  const double* k2ci;         // imaginary part of the cell k^2 (sponge) or null
};

template <typename R>
__global__ void fe3_assemble_kernel(FeMesh3 ms, cplx<R>* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= ms.nx || y >= ms.ny || z >= ms.nz) return;
  const int node[3] = {x, y, z};
  const int N[3] = {ms.nx, ms.ny, ms.nz};
  c128 acc[27];
  for (int q = 0; q < 27; ++q) acc[q] = mk(0.0, 0.0);
  for (int co = 0; co < 8; ++co) {
    int cell[3], corner[3];
    for (int l = 0; l < 3; ++l) {
      const int o = (co >> l) & 1;          // cell node (o = 0) or node + 1 (o = 1) along l
      cell[l] = node[l] + o;
      corner[l] = o == 0 ? 1 : 0;           // the node's corner index in that cell
    }
    const int gcx = min(max(cell[0] - ms.wl + ms.lo, ms.lo), ms.hi + 1);
    double kr;
    const c128 k2 =
        cell_k2(ms.k2c, ms.k2ci, ((size_t)cell[2] * ms.k2_ny1 + cell[1]) * ms.k2_ld + gcx, &kr);
    double hl[3];
    c128 al[3];
    for (int l = 0; l < 3; ++l) {
      hl[l] = ms.h[l][cell[l]];
      al[l] = ms.a[l][cell[l]];
    }
    double c[5];
    table9_3d(ms.H * kr / (2.0 * M_PI), c);
    const double I[4] = {c[0] / 8, c[1] / 24, c[2] / 24, (1 - c[0] - c[1] - c[2]) / 8};
    const double Jc[3] = {c[3] / 4, c[4] / 8, (1 - c[3] - c[4]) / 4};
    const c128 pa = al[0] * al[1] * al[2];
    const c128 mass = (hl[0] * hl[1] * hl[2] * k2) * cinv(pa);
    c128 stiff[3];                           // (alpha_l / h_l) prod_{m != l} (h_m / alpha_m)
    for (int l = 0; l < 3; ++l) {
      c128 v = (1.0 / hl[l]) * al[l];
      for (int m = 0; m < 3; ++m)
        if (m != l) v = hl[m] * (v * cinv(al[m]));
      stiff[l] = v;
    }
    for (int bo = 0; bo < 8; ++bo) {
      int nb[3], b[3];
      bool ok = true;
      for (int l = 0; l < 3; ++l) {
        b[l] = (bo >> l) & 1;
        nb[l] = cell[l] + b[l] - 1;          // neighbour unknown along l
        ok = ok && nb[l] >= 0 && nb[l] < N[l];
      }
      if (!ok) continue;
      int ham = 0;
      for (int l = 0; l < 3; ++l) ham += (corner[l] != b[l]);
      c128 v = -(I[ham] * mass);
      for (int l = 0; l < 3; ++l) {
        int hamo = 0;
        for (int m = 0; m < 3; ++m)
          if (m != l) hamo += (corner[m] != b[m]);
        const double sg = (corner[l] == b[l]) ? -1.0 : 1.0;
        v = v - (sg * Jc[hamo]) * stiff[l];
      }
      const int q = (nb[2] - z + 1) * 9 + (nb[1] - y + 1) * 3 + (nb[0] - x + 1);
      acc[q] = acc[q] + v;
    }
  }
  const size_t base = (size_t)z * ms.sz + (size_t)y * ms.sy + (size_t)x * ms.sx;
  for (int q = 0; q < 27; ++q) out[q * ms.sq + base] = ccast<R>(acc[q]);
}

// One axis of the transfer: restriction weights of coarse unknown q (coarse
// node Q = q + 1) on the fine unknowns i_FP(Q) - 2 + a, a = 0, 1, 2.
struct Tr1 {
  int u0;
  double w[3];
};
__device__ __forceinline__ Tr1 tr_axis(int q, const int* ifp, const int* refined) {
  const int Q = q + 1;
  Tr1 t;
  t.w[0] = refined[Q - 1] ? 0.5 : 0.0;
  t.w[1] = 1.0;
  t.w[2] = refined[Q] ? 0.5 : 0.0;
  t.u0 = ifp[Q] - 2;
  return t;
}

// r_c = P^T r_f (Section 4.2: R is the transpose of the prolongation); 2-D
// when ifpz is null.
template <typename R>
__global__ void restrict_kernel(int Ncx, int Ncy, int Ncz, int Nfx, int Nfy, int Nfz,
                                const int* ifpx, const int* refx, const int* ifpy,
                                const int* refy, const int* ifpz, const int* refz,
                                const cplx<R>* rf, cplx<R>* rc) {
  const int qx = blockIdx.x * blockDim.x + threadIdx.x;
  const int qy = blockIdx.y;
  const int qz = blockIdx.z % Ncz, r = blockIdx.z / Ncz;
  if (qx >= Ncx) return;
  const Tr1 tx = tr_axis(qx, ifpx, refx), ty = tr_axis(qy, ifpy, refy);
  Tr1 tz;
  if (ifpz) {
    tz = tr_axis(qz, ifpz, refz);
  } else {
    tz.u0 = -1;
    tz.w[0] = 0.0; tz.w[1] = 1.0; tz.w[2] = 0.0;
  }
  const size_t nf = (size_t)Nfx * Nfy * Nfz;
  const cplx<R>* f = rf + (size_t)r * nf;
  cplx<R> acc = mk<R>(0, 0);
  for (int c = 0; c < 3; ++c) {
    if (tz.w[c] == 0.0) continue;
    const int uz = tz.u0 + c;
    for (int a = 0; a < 3; ++a) {
      if (ty.w[a] == 0.0) continue;
      const int uy = ty.u0 + a;
      for (int b = 0; b < 3; ++b) {
        if (tx.w[b] == 0.0) continue;
        const int ux = tx.u0 + b;
        acc = acc + (R)(tz.w[c] * ty.w[a] * tx.w[b]) * f[((size_t)uz * Nfy + uy) * Nfx + ux];
      }
    }
  }
  rc[(size_t)r * Ncx * Ncy * Ncz + ((size_t)qz * Ncy + qy) * Ncx + qx] = acc;
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

// u_f += P e_c (2-D when q0z is null)
template <typename R>
__global__ void prolong_add_kernel(int Nfx, int Nfy, int Nfz, int ncx, int ncy, int ncz,
                                   const int* q0x, const int* q1x, const int* q0y,
                                   const int* q1y, const int* q0z, const int* q1z,
                                   const cplx<R>* ec, cplx<R>* uf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;   // fine unknown, node x + 1
  const int y = blockIdx.y;
  const int z = blockIdx.z % Nfz, r = blockIdx.z / Nfz;
  if (x >= Nfx) return;
  const int Ncx = ncx - 1, Ncy = ncy - 1, Ncz = q0z ? ncz - 1 : 1;
  const cplx<R>* e = ec + (size_t)r * Ncx * Ncy * Ncz;
  int sx[2] = {q0x[x + 1], q1x[x + 1]}, sy[2] = {q0y[y + 1], q1y[y + 1]};
  int sz[2] = {1, -1};
  if (q0z) { sz[0] = q0z[z + 1]; sz[1] = q1z[z + 1]; }
  const R wx = sx[1] >= 0 ? (R)0.5 : (R)1, wy = sy[1] >= 0 ? (R)0.5 : (R)1;
  const R wz = sz[1] >= 0 ? (R)0.5 : (R)1;
  cplx<R> v = mk<R>(0, 0);
  for (int c = 0; c < 2; ++c) {
    const int Qz = sz[c];
    if (Qz < 0) continue;
    if (q0z && (Qz <= 0 || Qz >= ncz)) continue;       // Dirichlet coarse nodes carry zero
    const int iz = q0z ? Qz - 1 : 0;
    for (int a = 0; a < 2; ++a) {
      const int Qy = sy[a];
      if (Qy < 0 || Qy <= 0 || Qy >= ncy) continue;
      for (int b = 0; b < 2; ++b) {
        const int Qx = sx[b];
        if (Qx < 0 || Qx <= 0 || Qx >= ncx) continue;
        v = v + (wz * wy * wx) * e[((size_t)iz * Ncy + (Qy - 1)) * Ncx + (Qx - 1)];
      }
    }
  }
  cplx<R>* u = uf + (size_t)r * Nfx * Nfy * Nfz + ((size_t)z * Nfy + y) * Nfx + x;
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

// n_int[l]: interior fine cells along x, y, z (z unused in 2-D).
void build_level_fe(hz_handle* h, Level& L, const Level& fine, const int* n_int, int w_out,
                    double hh, cudaStream_t s) {
  const int d = fine.dim3d ? 3 : 2;
  L.dim3d = fine.dim3d;
  // sponge: standard coarsening (Section 4.1), every fine cell merged in
  // pairs, no kept layers and no PML on the coarse grid
  const bool sponge = h->p.boundary == HZ_BOUNDARY_SPONGE;
  int n_in[3] = {n_int[0], n_int[1], d == 3 ? n_int[2] : 0};
  if (sponge) {
    for (int l = 0; l < d; ++l) n_in[l] += 2 * w_out;
    w_out = 0;
  }
  n_int = n_in;
  int n_c[3] = {1, 1, 1};
  for (int l = 0; l < d; ++l) n_c[l] = 2 * w_out + n_int[l] / 2;
  L.nx = n_c[0] - 1;
  L.ny = n_c[1] - 1;
  L.nz = d == 3 ? n_c[2] - 1 : 1;
  L.h = 2 * hh;                            // interior coarse spacing H
  L.fe = true;
  const double C = (w_out > 0) ? h->p.s_pml_out * h->c_pml / std::pow(w_out * hh, 3) : 0.0;
  AxisTables* axes[3] = {&L.ax, &L.ay, &L.az};
  const int Nf[3] = {fine.nx, fine.ny, fine.nz};
  for (int l = 0; l < d; ++l) {
    L.ifp[l] = (int*)dmalloc(sizeof(int) * (n_c[l] + 1));
    L.refined[l] = (int*)dmalloc(sizeof(int) * (n_c[l] + 1));
    AxisTables* a = axes[l];
    alloc_axis_fe(*a, n_c[l] - 1);
    coarse_axis_kernel<<<cdiv(n_c[l] + 1, 128), 128, 0, s>>>(
        n_c[l], w_out, n_int[l], hh, C, h->p.omega, a->a_node, a->a_cell, a->h_cell, a->a_node32,
        a->a_cell32, L.ifp[l], L.refined[l]);
    // prolongation maps (fine node -> coarse sources)
    const int nf_cells = 2 * w_out + n_int[l];
    L.q0[l] = (int*)dmalloc(sizeof(int) * (nf_cells + 1));
    L.q1[l] = (int*)dmalloc(sizeof(int) * (nf_cells + 1));
    prolong_map_kernel<<<cdiv(n_c[l] + 1, 128), 128, 0, s>>>(n_c[l], L.ifp[l], L.refined[l],
                                                              L.q0[l], L.q1[l]);
  }
  const int ncz = d == 3 ? n_c[2] : 1;
  const size_t ncells = (size_t)n_c[0] * n_c[1] * ncz;
  L.k2c = (double*)dmalloc(sizeof(double) * ncells);
  if (sponge) L.k2ci = (double*)dmalloc(sizeof(double) * ncells);
  coarse_k2_kernel<<<dim3(cdiv(n_c[0], 128), n_c[1], ncz), 128, 0, s>>>(
      n_c[0], n_c[1], ncz, Nf[0], Nf[1], Nf[2], L.ifp[0], L.refined[0], L.ifp[1], L.refined[1],
      L.ifp[2], L.refined[2], fine.m, h->p.omega * h->p.omega, L.k2c, fine.ax.beta,
      fine.ay.beta, d == 3 ? fine.az.beta : nullptr, L.k2ci);
  const size_t plane = L.size();
  const int nq = L.planes();
  L.st128 = (c128*)dmalloc(sizeof(c128) * nq * plane);
  L.st64 = (c64*)dmalloc(sizeof(c64) * nq * plane);
  if (d == 2) {
    FeMesh ms{L.nx, L.ny, L.ax.h_cell, L.ax.a_cell, L.ay.h_cell, L.ay.a_cell, L.k2c, n_c[0],
              0, L.nx - 1, 0, L.h, h->p.omega, plane, (size_t)L.nx, 1, L.k2ci};
    dim3 grid(cdiv(L.nx, 128), L.ny);
    fe_assemble_kernel<double><<<grid, 128, 0, s>>>(ms, L.st128);
    fe_assemble_kernel<float><<<grid, 128, 0, s>>>(ms, L.st64);
  } else {
    FeMesh3 ms{L.nx, L.ny, L.nz, {L.ax.h_cell, L.ay.h_cell, L.az.h_cell},
               {L.ax.a_cell, L.ay.a_cell, L.az.a_cell}, L.k2c, n_c[0], n_c[1], 0, L.nx - 1, 0,
               L.h, h->p.omega, plane, (size_t)L.nx * L.ny, (size_t)L.nx, 1, L.k2ci};
    dim3 grid(cdiv(L.nx, 64), L.ny, L.nz);
    fe3_assemble_kernel<double><<<grid, 64, 0, s>>>(ms, L.st128);
    fe3_assemble_kernel<float><<<grid, 64, 0, s>>>(ms, L.st64);
  }
  HZ_CU(cudaGetLastError());
  HZ_CU(cudaStreamSynchronize(s));
}

// Slab stencil of the coarse FE operator on the extended slab mesh: cell k^2
// frozen to the interface cell in the added PML (Eq. 10, cellwise).  2-D:
// st [ny][9][wp]; 3-D: st3 [nz][27][ny][W].
template <typename R>
void slab_stencil_fe(hz_handle* h, const Level& L, const Slab& S, cudaStream_t s) {
  if (!L.dim3d) {
    FeMesh ms{S.W, L.ny, S.ax.h_cell, S.ax.a_cell, L.ay.h_cell, L.ay.a_cell, L.k2c, L.nx + 1,
              S.lo, S.hi, S.wl, L.h, h->p.omega, (size_t)S.wp, (size_t)9 * S.wp, 1, L.k2ci};
    dim3 grid(cdiv(S.W, 128), L.ny);
    fe_assemble_kernel<R><<<grid, 128, 0, s>>>(ms, (cplx<R>*)S.st);
  } else {
    const size_t B = (size_t)L.ny * S.W;
    FeMesh3 ms{S.W, L.ny, L.nz, {S.ax.h_cell, L.ay.h_cell, L.az.h_cell},
               {S.ax.a_cell, L.ay.a_cell, L.az.a_cell}, L.k2c, L.nx + 1, L.ny + 1, S.lo, S.hi,
               S.wl, L.h, h->p.omega, B, 27 * B, (size_t)S.W, 1, L.k2ci};
    dim3 grid(cdiv(S.W, 64), L.ny, L.nz);
    fe3_assemble_kernel<R><<<grid, 64, 0, s>>>(ms, (cplx<R>*)S.st3);
  }
  HZ_CU(cudaGetLastError());
}

template <typename R>
void restrict_residual(hz_handle* h, const Level& F, const Level& C, const cplx<R>* rf,
                       cplx<R>* rc, int n_rhs, cudaStream_t s) {
  dim3 grid(cdiv(C.nx, 128), C.ny, C.nz * n_rhs);
  restrict_kernel<R><<<grid, 128, 0, s>>>(C.nx, C.ny, C.nz, F.nx, F.ny, F.nz, C.ifp[0],
                                          C.refined[0], C.ifp[1], C.refined[1], C.ifp[2],
                                          C.refined[2], rf, rc);
  h->launches++;
  HZ_CU(cudaGetLastError());
}

template <typename R>
void prolong_add(hz_handle* h, const Level& F, const Level& C, const cplx<R>* ec, cplx<R>* uf,
                 int n_rhs, cudaStream_t s) {
  dim3 grid(cdiv(F.nx, 128), F.ny, F.nz * n_rhs);
  prolong_add_kernel<R><<<grid, 128, 0, s>>>(F.nx, F.ny, F.nz, C.nx + 1, C.ny + 1, C.nz + 1,
                                             C.q0[0], C.q1[0], C.q0[1], C.q1[1], C.q0[2],
                                             C.q1[2], ec, uf);
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
template void prolong_add<double>(hz_handle*, const Level&, const Level&, const c128*, c128*,
                                  int, cudaStream_t);

}  // namespace hz
