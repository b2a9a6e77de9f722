// 3-D slabs: set-up, factorisation and solves of the subdomain operators
// A^(j) (SubdomSolve, Table 2; the paper factors them with a sparse direct
// solver on CPU process groups, Section 5).
//
// A 3-D slab (x width W, all of y and z) is block tridiagonal along z: block
// row k is the z layer k with B = N_y W unknowns (index b = y W + e).  D_k
// couples a layer to itself (5-point in (y, x) for finite differences, 9-point
// for the coarse FE operator), the couplings to the layers k -/+ 1 are
// diagonal (7-point) or 9-point (27-point FE).  The slab stencil is stored
// as 27 planes per layer, q = (dz+1) 9 + (dy+1) 3 + (dx+1).
//
// Twisted block LU, as for the 2-D slabs: a chain from layer 0 and a chain
// from layer nz-1 meet at layer m = (nz-1)/2:
//   S_t = D_{k_t} - L_t G_{t-1} R_{t-1},  G_t = S_t^-1,
//   S_m = D_m - C_m G_{m-1} B_{m-1} - B_m G_{m+1} C_{m+1},
// with L_t / R_t the couplings of a layer to the previous / next layer of its
// chain.  The blocks are dense (B ~ 10^3 - 4 10^3): each inverse is a blocked
// Gauss-Jordan elimination with implicit partial pivoting (pivot rows are
// marked, not moved; G[p][piv[q]] = S[piv[p]][q] at the end).  One
// elimination step with pivot row r for column p is the rank-1 update
//   S -= c rho^T,  c = S[:, p] - e_r,  rho = S[r, :] / S[r][p] + e_p,
// which turns column p into the inverse's column.  Two levels of blocking:
// within an outer block of KO columns (hz_params.block_3d), panels of 16 (or NB) columns: one
// CTA per chain eliminates the panel's columns on the panel only and records
// the colmods c (C, B x KO), the pivot rows and 1 / S[r][p]; the pivot
// rows' other columns follow from the short recurrence
//   rho_t = (S[r_t, :] - sum_{s<t} C[r_t][s] rho_s) / S[r_t][p_t]
// (for columns outside the outer block with all earlier steps of the block,
// since those columns are not updated until the block ends); S -= C R then
// updates the block's other columns (rank 16), and at the end of the block
// all columns outside it (a dense complex GEMM of depth KO, on the tensor
// cores in complex64).  Every launch takes all chains of all slabs at the
// same step.
//
// Solve: forward y_t = G_t (f_t - L_t y_{t-1}) along both chains, meeting
// x_m = G_m (f_m - C_m y_{m-1} - B_m y_{m+1}), backward
// x_t = y_t - G_t R_t x_{t+1}: per layer one sparse coupling apply and one
// dense GEMV with the stored inverse (a skinny GEMM over the right-hand
// sides).
#include "hz_internal.h"
#include "ptx.cuh"
#include "tc.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

namespace hz {

namespace {

// Programmatic dependent launch: the solve kernels are launched with
// programmatic stream serialisation, so a kernel's launch and block set-up
// overlap its predecessor; every such kernel waits for the predecessor's
// results (griddepcontrol.wait) before touching any data.
__device__ __forceinline__ void pdl_wait3() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
void launch_pdl3s(void (*k)(KArgs...), dim3 grid, unsigned block, size_t smem, cudaStream_t s,
                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  HZ_CU(cudaLaunchKernelEx(&cfg, k, args...));
}

template <typename... KArgs, typename... Args>
void launch_pdl3(void (*k)(KArgs...), dim3 grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  HZ_CU(cudaLaunchKernelEx(&cfg, k, args...));
}

constexpr int NB = 32;            // panel width of the blocked Gauss-Jordan inverse
constexpr int kOuterDefault = 128;  // outer block of panels (rank of the delayed update);
constexpr int kOuterMax = 256;      //   hz_params.block_3d: 64, 128 or 256
constexpr int kPanelThreads = 512;
constexpr int kMaxB = 8192;       // largest block (pivot flags live in shared memory)
constexpr int kG3MaxSplit = 16;   // split-K ranges of the layer GEMM (many right-hand sides)

template <typename R>
__device__ __forceinline__ cplx<R> ldg(const cplx<R>* p) { return *p; }

// plane index of the coupling (dz, dy, dx)
__host__ __device__ __forceinline__ int qidx(int dz, int dy, int dx) {
  return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}

// ------------------------------------------------------------------ set-up
// Slab stencil of the 7-point operator (Eq. 40 in 3-D, times h^3) on the
// extended slab mesh, k frozen to the adjacent core column in the added PML
// (Eq. 10).  st3[k][q][y][e]; couplings to Dirichlet nodes are zero.
template <typename R>
__global__ void slab3_stencil_fd_kernel(int W, int ny, int nz, int lo, int hi, int wl, int nx,
                                        double hh, double h2w2, const double* m,
                                        const c128* sa_node, const c128* sa_cell,
                                        const c128* ay_node, const c128* ay_cell,
                                        const c128* az_node, const c128* az_cell,
                                        const double* bx, const double* by, const double* bz,
                                        cplx<R>* st) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (e >= W) return;
  const int g = min(max(e - wl + lo, lo), hi);
  const double mm = m[((size_t)z * ny + y) * nx + g];
  const c128 i1 = cinv(sa_node[e]), i2 = cinv(ay_node[y]), i3 = cinv(az_node[z]);
  const c128 s23 = i2 * i3, s13 = i1 * i3, s12 = i1 * i2;
  const c128 xl = sa_cell[e], xr = sa_cell[e + 1];
  const c128 yl = ay_cell[y], yr = ay_cell[y + 1];
  const c128 zl = az_cell[z], zr = az_cell[z + 1];
  const c128 zero = mk(0.0, 0.0);
  c128 v[27];
  for (int q = 0; q < 27; ++q) v[q] = zero;
  // sponge: k^2 (1 + i beta)^2, frozen with k in the added columns (Eq. 10)
  const c128 sp = bx ? sponge_s(bx[g] + by[y] + bz[z]) : mk(1.0, 0.0);
  v[qidx(0, 0, 0)] = hh * (s23 * (xl + xr) + s13 * (yl + yr) + s12 * (zl + zr)) -
                     (hh * h2w2 * mm) * (sp * (s12 * i3));
  if (e > 0) v[qidx(0, 0, -1)] = -(hh * (s23 * xl));
  if (e < W - 1) v[qidx(0, 0, 1)] = -(hh * (s23 * xr));
  if (y > 0) v[qidx(0, -1, 0)] = -(hh * (s13 * yl));
  if (y < ny - 1) v[qidx(0, 1, 0)] = -(hh * (s13 * yr));
  if (z > 0) v[qidx(-1, 0, 0)] = -(hh * (s12 * zl));
  if (z < nz - 1) v[qidx(1, 0, 0)] = -(hh * (s12 * zr));
  const size_t B = (size_t)ny * W;
  cplx<R>* out = st + (size_t)z * 27 * B + (size_t)y * W + e;
  for (int q = 0; q < 27; ++q) out[(size_t)q * B] = ccast<R>(v[q]);
}

// Transmission coefficients of Eqs. 19-20 (global A entries between the two
// layers of columns), per (z, y) and transverse offset t = (dz+1) 3 + (dy+1):
//   inj[0] = +A_{beta,beta+1} (multiplies B[1]), inj[1] = -A_{beta+1,beta} (B[0]),
//   inj[2] = -A_{bt,bt+1} (B[1]),                inj[3] = +A_{bt+1,bt} (B[0]),
// beta = beta_{j-1}, bt = tilde-beta_j (-1: no such neighbour).  Finite
// differences: only t = 4 (dz = dy = 0), A_{x,x+1} = -h alpha_{x+1/2} / (alpha_y alpha_z);
// FE: read from the level's 27 stored planes.
template <typename R>
__global__ void inj3_kernel(int nx, int ny, int nz, int beta, int bt, double hh,
                            const c128* ax_cell, const c128* ay_node, const c128* az_node,
                            const c128* st, cplx<R>* inj) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (y >= ny) return;
  const size_t plane = (size_t)nx * ny * nz;
  const size_t row = ((size_t)z * ny + y);
  const size_t nt = (size_t)ny * nz;
  const c128 zero = mk(0.0, 0.0);
  for (int t = 0; t < 9; ++t) {
    const int dz = t / 3 - 1, dy = t % 3 - 1;
    c128 f0 = zero, f1 = zero, b0 = zero, b1 = zero;
    if (st) {
      if (beta >= 0) {
        f0 = st[(size_t)qidx(dz, dy, 1) * plane + row * nx + beta];
        f1 = -st[(size_t)qidx(dz, dy, -1) * plane + row * nx + beta + 1];
      }
      if (bt >= 0) {
        b0 = -st[(size_t)qidx(dz, dy, 1) * plane + row * nx + bt];
        b1 = st[(size_t)qidx(dz, dy, -1) * plane + row * nx + bt + 1];
      }
    } else if (t == 4) {
      const c128 s = hh * cinv(ay_node[y] * az_node[z]);
      const c128 af = beta >= 0 ? -(s * ax_cell[beta + 1]) : zero;
      const c128 ab = bt >= 0 ? -(s * ax_cell[bt + 1]) : zero;
      f0 = af; f1 = -af; b0 = -ab; b1 = ab;
    }
    const c128 vals[4] = {f0, f1, b0, b1};
    for (int q = 0; q < 4; ++q) inj[((size_t)q * nt + row) * 9 + t] = ccast<R>(vals[q]);
  }
}

}  // namespace

template <typename R>
void build_slabs3d(hz_handle* h, Level& L, cudaStream_t s) {
  L.slabs.assign(L.J + 1, Slab{});
  if (L.nz < 3) throw Failure(HZ_EINVAL, "a 3-D slab needs at least 3 z layers");
  const size_t el = sizeof(cplx<R>);
  const int R_ = h->p.max_rhs;
  for (int j = 1; j <= L.J; ++j) {
    Slab& S = L.slabs[j];
    slab_geometry(h, L, S, j, s);
    S.B = L.ny * S.W;
    if (S.B > kMaxB)
      throw Failure(HZ_EINVAL, "3-D slab block too large (N_y W = " + std::to_string(S.B) +
                                   " > " + std::to_string(kMaxB) + ")");
    S.bstride = ((size_t)S.B * S.B + 15) / 16 * 16;
    const size_t B = S.B;
    S.st3 = dmalloc(el * (size_t)L.nz * 27 * B);
    HZ_CU(cudaMemsetAsync(S.st3, 0, el * (size_t)L.nz * 27 * B, s));
    S.inj3 = dmalloc(el * 4 * L.nt() * 9);
    const int beta = (j > 1) ? L.beta[j - 1] : -1;
    const int bt = (j < L.J) ? L.beta_t[j] : -1;
    if (!L.fe) {
      const double h2w2 = L.h * L.h * h->p.omega * h->p.omega;
      slab3_stencil_fd_kernel<R><<<dim3(cdiv(S.W, 64), L.ny, L.nz), 64, 0, s>>>(
          S.W, L.ny, L.nz, S.lo, S.hi, S.wl, L.nx, L.h, h2w2, L.m, S.ax.a_node, S.ax.a_cell,
          L.ay.a_node, L.ay.a_cell, L.az.a_node, L.az.a_cell, L.ax.beta, L.ay.beta, L.az.beta,
          (cplx<R>*)S.st3);
      inj3_kernel<R><<<dim3(cdiv(L.ny, 128), L.nz), 128, 0, s>>>(
          L.nx, L.ny, L.nz, beta, bt, L.h, L.ax.a_cell, L.ay.a_node, L.az.a_node, nullptr,
          (cplx<R>*)S.inj3);
    } else {
      slab_stencil_fe<R>(h, L, S, s);
      inj3_kernel<R><<<dim3(cdiv(L.ny, 128), L.nz), 128, 0, s>>>(
          L.nx, L.ny, L.nz, beta, bt, L.h, nullptr, nullptr, nullptr, L.st128, (cplx<R>*)S.inj3);
    }
    HZ_CU(cudaGetLastError());
    S.G = dmalloc(el * S.bstride * L.nz);
    S.Y = dmalloc(el * (size_t)L.nz * R_ * B);
    S.V = dmalloc(el * 2 * (size_t)R_ * B);
    if (R_ > 4) S.gpart = dmalloc(el * 2 * kG3MaxSplit * (size_t)R_ * B);
    if (R_ > 4 && sizeof(R) == 4) {
      // packed inverses for the tensor-core layer products (zero padding kept)
      const size_t nrt = cdiv(B, 128), nkc = cdiv(B, 16);
      S.gp_layer = nrt * nkc * 8192;
      S.Gp = (float*)dmalloc(sizeof(float) * S.gp_layer * L.nz);
      HZ_CU(cudaMemsetAsync(S.Gp, 0, sizeof(float) * S.gp_layer * L.nz, s));
      S.Vp = (float*)dmalloc(sizeof(float) * 2 * nkc * 2048);
      // zero padding (rows beyond B of the last chunk): the products with
      // at most 32 right-hand sides write only the live entries
      HZ_CU(cudaMemsetAsync(S.Vp, 0, sizeof(float) * 2 * nkc * 2048, s));
    }
  }
  L.mid = (L.nz - 1) / 2;
  HZ_CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ factorisation
namespace {

// One elimination chain at one step (or the meeting layer of a slab): the
// layer k to factor, the Schur terms (previous layers kp with the dz of the
// coupling k -> kp (L) and kp -> k (R)), the slab's stencil and inverses, and
// the chain's work buffers.
template <typename R>
struct FChain {
  int B, W, ny;
  int k, nterm;
  int kp[2], dzL[2], dzR[2];
  const cplx<R>* st;   // [nz][27][B]
  cplx<R>* G;          // [nz][bstride]
  size_t bstride;
  cplx<R>* S;          // [B][B] Schur complement, inverted in place
  cplx<R>* C;          // [KO][B] colmods of the current outer block (slot = column - P0)
  cplx<R>* Rm;         // [KO][B] rowmods of the current outer block
  cplx<R>* pinfo;      // [KO] 1 / pivot of the block's columns
  int* piv;            // [B] pivot row of column p
  int* pinv;           // [B] column whose pivot row is r (-1: not yet a pivot row)
  int* prow;           // [KO] pivot rows of the block's columns
  float* Ap;           // complex64 tensor-core path: packed colmods (tc_pack_kernel)
  float* Bp;           //   and rowmods of the current outer block
  float* Gp;           // packed inverses of the slab's layers (layer stride gp_layer) or null
  size_t gp_layer;
};

// Entry (i, j) of the in-layer block D_k (9-point in (y, x), zero elsewhere).
template <typename R>
__device__ __forceinline__ cplx<R> d_entry(const FChain<R>& c, int i, int j) {
  const int W = c.W;
  const int yi = i / W, ei = i - yi * W, yj = j / W, ej = j - yj * W;
  const int dy = yj - yi, dx = ej - ei;
  if (dy < -1 || dy > 1 || dx < -1 || dx > 1) return mk<R>(0, 0);
  return c.st[((size_t)c.k * 27 + qidx(0, dy, dx)) * c.B + i];
}

// T = G_kp R (term `term`): T[a][j] = sum_{(dy,dx)} G_kp[a][b] R_{(dy,dx)}[b],
// b = j - (dy W + dx) the row of R that couples to column j; written into
// the G slot of layer k (free until its inverse is written).
template <typename R>
__global__ void __launch_bounds__(128) schur_T_kernel(const FChain<R>* chains, int term) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.z];
  const int j = blockIdx.x * blockDim.x + threadIdx.x, a = blockIdx.y;
  if (j >= c.B || a >= c.B) return;
  const int W = c.W, yj = j / W, ej = j - yj * W;
  // static indices into the descriptor's two-term arrays (a runtime index
  // would copy the descriptor to local memory in every thread)
  const int kp = term == 0 ? c.kp[0] : c.kp[1], dzR = term == 0 ? c.dzR[0] : c.dzR[1];
  const cplx<R>* Gp = c.G + (size_t)kp * c.bstride + (size_t)a * c.B;
  const cplx<R>* stp = c.st + (size_t)kp * 27 * c.B;
  cplx<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int yb = yj - dy;
    if (yb < 0 || yb >= c.ny) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int eb = ej - dx;
      if (eb < 0 || eb >= W) continue;
      const int b = yb * W + eb;
      cfma(acc, Gp[b], stp[(size_t)qidx(dzR, dy, dx) * c.B + b]);
    }
  }
  c.G[(size_t)c.k * c.bstride + (size_t)a * c.B + j] = acc;
}

// S[i][j] = (init ? D[i][j] : S[i][j]) - Schur terms.  Finite differences
// (fe = 0, diagonal couplings): every term, l_i G_kp[i][j] r_j, directly.
// FE: the one term `term` from T (schur_T_kernel) in the G slot of layer k:
// sum_{(dy,dx)} L_{(dy,dx)}[i] T[i + dy W + dx][j].  Also marks every row as
// not yet a pivot row (init).
template <typename R>
__global__ void __launch_bounds__(128) schur_S_kernel(const FChain<R>* chains, int term, int init,
                                                      int fe) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.z];
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= c.B || i >= c.B) return;
  if (init && j == 0) c.pinv[i] = -1;
  cplx<R>* Sij = c.S + (size_t)i * c.B + j;
  cplx<R> v = init ? d_entry(c, i, j) : *Sij;
  const cplx<R>* stk = c.st + (size_t)c.k * 27 * c.B;
  if (!fe) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {   // static indices into the two-term arrays
      if (t >= c.nterm) break;
      const cplx<R> l = stk[(size_t)qidx(c.dzL[t], 0, 0) * c.B + i];
      const cplx<R> r = c.st[((size_t)c.kp[t] * 27 + qidx(c.dzR[t], 0, 0)) * c.B + j];
      const cplx<R> g = c.G[(size_t)c.kp[t] * c.bstride + (size_t)i * c.B + j];
      v = v - l * (g * r);
    }
  } else if (term >= 0) {
    const int W = c.W, yi = i / W, ei = i - yi * W;
    const int dzL = term == 0 ? c.dzL[0] : c.dzL[1];
    const cplx<R>* T = c.G + (size_t)c.k * c.bstride;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int ya = yi + dy;
      if (ya < 0 || ya >= c.ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ea = ei + dx;
        if (ea < 0 || ea >= W) continue;
        const cplx<R> l = stk[(size_t)qidx(dzL, dy, dx) * c.B + i];
        v = v - l * T[(size_t)(ya * W + ea) * c.B + j];
      }
    }
  }
  *Sij = v;
}

// Pivot key: unpivoted rows rank by |v|^2 (float bits, monotone for
// non-negative values), ties to the lowest row; pivoted rows are 0, so an
// unpivoted row always wins (also for NaN or zero columns).
__device__ __forceinline__ unsigned long long pivot_key(float a2, int row) {
  const unsigned int bits = __float_as_uint(a2) & 0x7fffffffu;
  return ((unsigned long long)(bits + 1u) << 32) | (unsigned long long)(0xffffffffu - (unsigned)row);
}

// Panel [p0, p0 + nbp) of the Gauss-Jordan inverse of one chain's S (one CTA
// per chain): lane q of a warp holds column p0 + q of a row; warp w takes rows
// w, w + 16, ...  Each step chooses the pivot row of column p0 + t, forms its
// scaled panel row, and applies the rank-1 update to the panel columns of
// every row, recording the colmods (C) and the next column's pivot keys.
template <typename R>
__global__ void __launch_bounds__(kPanelThreads) gj_panel_kernel(const FChain<R>* chains, int p0,
                                                                 int slot) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.x];
  const int B = c.B;
  if (p0 >= B) return;
  const int nbp = min(NB, B - p0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kPanelThreads / 32;
  __shared__ unsigned char flag[kMaxB];
  __shared__ unsigned long long wkey[NW];
  __shared__ cplx<R> rm[NB];
  __shared__ int sh_r;
  for (int i = threadIdx.x; i < B; i += kPanelThreads) flag[i] = c.pinv[i] >= 0;
  __syncthreads();
  // keys of column p0
  unsigned long long best = 0;
  for (int i = warp; i < B; i += NW) {
    const cplx<R> v = lane == 0 ? c.S[(size_t)i * B + p0] : mk<R>(0, 0);
    if (lane == 0 && !flag[i]) {
      const unsigned long long k = pivot_key((float)cabs2(v), i);
      best = k > best ? k : best;
    }
  }
  for (int t = 0; t < nbp; ++t) {
    if (lane == 0) wkey[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long b = 0;
      for (int w = 0; w < NW; ++w) b = wkey[w] > b ? wkey[w] : b;
      const int r = (int)(0xffffffffu - (unsigned)(b & 0xffffffffu));
      sh_r = r;
      flag[r] = 1;
      c.piv[p0 + t] = r;
      c.pinv[r] = p0 + t;
      c.prow[slot + t] = r;
    }
    __syncthreads();
    const int r = sh_r;
    if (warp == 0) {
      const cplx<R> v = lane < nbp ? c.S[(size_t)r * B + p0 + lane] : mk<R>(0, 0);
      const cplx<R> pv = mk<R>(__shfl_sync(0xffffffffu, v.re, t), __shfl_sync(0xffffffffu, v.im, t));
      const cplx<R> inv = cinv(pv);
      cplx<R> x = v * inv;
      if (lane == t) x = inv + mk<R>(1, 0);
      if (lane < NB) rm[lane] = x;
      if (lane == 0) c.pinfo[slot + t] = inv;
    }
    __syncthreads();
    const cplx<R> rq = lane < nbp ? rm[lane] : mk<R>(0, 0);
    best = 0;
    for (int i = warp; i < B; i += NW) {
      cplx<R>* row = c.S + (size_t)i * B + p0;
      cplx<R> v = lane < nbp ? row[lane] : mk<R>(0, 0);
      cplx<R> ci = mk<R>(__shfl_sync(0xffffffffu, v.re, t), __shfl_sync(0xffffffffu, v.im, t));
      if (i == r) ci.re -= (R)1;
      v = v - ci * rq;
      if (lane < nbp) row[lane] = v;
      if (lane == 0) c.C[(size_t)(slot + t) * B + i] = ci;
      if (t + 1 < nbp) {
        const cplx<R> nv = mk<R>(__shfl_sync(0xffffffffu, v.re, t + 1),
                                 __shfl_sync(0xffffffffu, v.im, t + 1));
        if (lane == 0 && !flag[i]) {
          const unsigned long long k = pivot_key((float)cabs2(nv), i);
          best = k > best ? k : best;
        }
      }
    }
    __syncthreads();
  }
}

// The same panel elimination with the panel held in shared memory (blocks
// small enough: B x LD elements, B < 2047; complex128, and complex64 blocks
// too large for the register form below): rows tid, tid + 1024, ... per
// thread, panel rows padded to LD = PW + 1 elements (an odd stride).  Two
// block barriers per pivot:
//  * each warp reduces its 32-bit pivot keys (redux.sync) into its key slot;
//    after the first barrier every warp reduces the 32 slots itself, so that
//    all threads know the pivot row r, and the first warp writes the scaled
//    pivot row rho = S[r, :] / S[r][t] + e_t to shared memory;
//  * after the second barrier every thread applies the rank-1 step
//    row -= c_i rho to its rows (c_i = row[t], minus 1 on row r) and forms
//    their keys for column t + 1.
// The panel is loaded with cp.async (all of a thread's copies in flight at
// once); the colmods go to C [KO][B] at the panel's slots.
constexpr int kSmemPanelThreads = 1024;
static_assert(kSmemPanelThreads == 32 * 32, "one key slot per warp, each warp reduces all slots");

// 32-bit pivot key: the top 21 bits of |a|^2 (its exponent and leading 13
// mantissa bits) above the reversed row index (11 bits, rows < 2047), so that
// an unsigned maximum takes the largest magnitude, near-ties (within 2^-13)
// going to the lowest row; every candidate's key is nonzero.
__device__ __forceinline__ unsigned pivot_key32(float a2, int row) {
  return ((__float_as_uint(a2) & 0x7fffffffu) >> 10 << 11) | (2047u - (unsigned)row);
}

template <typename R>
__device__ __forceinline__ void cp_async_el3(cplx<R>* dst, const cplx<R>* src) {
  if constexpr (sizeof(cplx<R>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// row[q] -= s pr[q], q < PW, for one padded panel row (4 FMAs per element);
// pr is a separate buffer, so that the loads of both can run ahead of the
// stores
template <typename R, int PW, int LD>
__device__ __forceinline__ void panel_row_update(cplx<R>* __restrict__ row,
                                                 const cplx<R>* __restrict__ pr, cplx<R> s) {
  if constexpr (sizeof(R) == 4 && LD % 2 == 0) {
    float4* rv = reinterpret_cast<float4*>(row);
    const float4* pv = reinterpret_cast<const float4*>(pr);
#pragma unroll
    for (int h = 0; h < PW / 2; ++h) {
      float4 a = rv[h];
      const float4 b = pv[h];
      a.x = fmaf(-s.re, b.x, fmaf(s.im, b.y, a.x));
      a.y = fmaf(-s.re, b.y, fmaf(-s.im, b.x, a.y));
      a.z = fmaf(-s.re, b.z, fmaf(s.im, b.w, a.z));
      a.w = fmaf(-s.re, b.w, fmaf(-s.im, b.z, a.w));
      rv[h] = a;
    }
  } else {
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      cplx<R> a = row[q];
      const cplx<R> b = pr[q];
      a.re = fma(-s.re, b.re, fma(s.im, b.im, a.re));
      a.im = fma(-s.re, b.im, fma(-s.im, b.re, a.im));
      row[q] = a;
    }
  }
}

template <typename R, int PW, int LD>
__global__ void __launch_bounds__(kSmemPanelThreads) gj_panel_smem_kernel(const FChain<R>* chains,
                                                                         int p0, int slot) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.x];
  const int B = c.B;
  if (p0 >= B) return;
  const int nbp = min(PW, B - p0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* P = (cplx<R>*)smem_raw;                          // [B][LD]
  cplx<R>* rho = P + (size_t)B * LD;                        // [LD] scaled pivot row
  unsigned* wkey = (unsigned*)(rho + LD);                   // [32]
  unsigned char* flag = (unsigned char*)(wkey + 32);        // [B]
  for (int e = tid; e < B * PW; e += kSmemPanelThreads) {
    const int i = e / PW, q = e - i * PW;
    if (q < nbp)
      cp_async_el3(P + i * LD + q, c.S + (size_t)i * B + p0 + q);
    else
      P[i * LD + q] = mk<R>(0, 0);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  for (int i = tid; i < B; i += kSmemPanelThreads) flag[i] = c.pinv[i] >= 0;
  __syncthreads();
  unsigned best = 0;
  for (int i = tid; i < B; i += kSmemPanelThreads)
    if (!flag[i]) best = max(best, pivot_key32((float)cabs2(P[i * LD]), i));
  for (int t = 0; t < nbp; ++t) {
    best = __reduce_max_sync(0xffffffffu, best);
    if (lane == 0) wkey[warp] = best;
    __syncthreads();
    const unsigned kb = __reduce_max_sync(0xffffffffu, wkey[lane]);
    const int r = min(2047 - (int)(kb & 2047u), B - 1);
    if (warp == 0 && lane < PW) {   // the scaled pivot row, one element per lane
      const cplx<R>* pr = P + r * LD;
      const cplx<R> inv = cinv(pr[t]);
      rho[lane] = lane == t ? inv + mk<R>(1, 0) : pr[lane] * inv;
      if (lane == 0) {
        flag[r] = 1;
        c.piv[p0 + t] = r;
        c.pinv[r] = p0 + t;
        c.prow[slot + t] = r;
        c.pinfo[slot + t] = inv;
      }
    }
    __syncthreads();
    best = 0;
    for (int i = tid; i < B; i += kSmemPanelThreads) {
      cplx<R>* row = P + i * LD;
      cplx<R> ci = row[t];
      if (i == r) ci.re -= (R)1;
      c.C[(size_t)(slot + t) * B + i] = ci;
      panel_row_update<R, PW, LD>(row, rho, ci);
      // the vector stores above and the element load below touch the same
      // words: keep the compiler from reordering them
      asm volatile("" ::: "memory");
      if (t + 1 < nbp && !flag[i]) best = max(best, pivot_key32((float)cabs2(row[t + 1]), i));
    }
  }
  __syncthreads();
  for (int e = tid; e < B * PW; e += kSmemPanelThreads) {
    const int i = e / PW, q = e - i * PW;
    if (q < nbp) c.S[(size_t)i * B + p0 + q] = P[i * LD + q];
  }
}

template <typename R, int PW, int LD>
size_t panel_smem_bytes(int B) {
  return (size_t)(B + 1) * LD * sizeof(cplx<R>) + 32 * sizeof(unsigned) + B + 16;
}

template <int PW>
size_t panel_reg_smem_bytes(int B) {
  return (size_t)(B + 1) * (PW + 2) * sizeof(c64) + 32 * sizeof(unsigned) +
         PW * (sizeof(c64) + sizeof(int)) + B + 16;
}

// complex64 panel elimination with rows held in registers.  The
// shared-memory form above re-reads and re-writes the whole B x PW panel in
// shared memory at every pivot, which its shared-memory bandwidth bounds;
// here rows tid, tid + T, ..., tid + (NR - 1) T of each of the T threads stay
// in registers for all PW steps (T = 512 with two rows, or 448 with three
// for blocks of up to 1344 rows), and only rows from NR T on are updated in
// shared memory.  The step loop is not unrolled (one copy of its body stays
// in the instruction cache); the register rows' column t + 1, which gives
// the next pivot key and the next colmod, is picked out during the update by
// selects.  Two barriers per pivot as above: the warps reduce the pivot keys,
// the thread holding row r writes rho = S[r, :] / S[r][t] + e_t to shared
// memory, and every thread applies row -= c_i rho to its rows.  Shared
// memory stages the panel in and out (coalesced), holds the rows beyond NR T
// (padded to PW + 2 elements: 144-byte rows put eight consecutive rows'
// 16-byte accesses on disjoint banks), and the pivot bookkeeping is written
// out at the end.
template <int PW, int T, int NR>
__global__ void __launch_bounds__(T) gj_panel_reg_kernel(const FChain<float>* chains, int p0,
                                                         int slot) {
  constexpr int LD = PW + 2, NW = T / 32;
  static_assert(PW % 2 == 0 && T % 32 == 0 && NW <= 32, "float4 pairs; one key slot per warp");
  pdl_wait3();
  const FChain<float> c = chains[blockIdx.x];
  const int B = c.B;
  if (p0 >= B) return;
  const int nbp = min(PW, B - p0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c64* P = (c64*)smem_raw;                                  // [B][LD]
  c64* rho = P + (size_t)B * LD;                            // [LD]
  unsigned* wkey = (unsigned*)(rho + LD);                   // [32]
  c64* sinv = (c64*)(wkey + 32);                            // [PW] 1 / pivot
  int* spiv = (int*)(sinv + PW);                            // [PW] pivot rows
  unsigned char* flag = (unsigned char*)(spiv + PW);        // [B] rows from NR T on
  for (int e = tid; e < B * PW; e += T) {
    const int i = e / PW, q = e - i * PW;
    if (q < nbp)
      cp_async_el3(P + i * LD + q, c.S + (size_t)i * B + p0 + q);
    else
      P[i * LD + q] = mk<float>(0, 0);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  bool fl[NR];                           // not (or no longer) a pivot candidate
#pragma unroll
  for (int k = 0; k < NR; ++k) fl[k] = tid + k * T >= B || c.pinv[tid + k * T] >= 0;
  for (int i = tid + NR * T; i < B; i += T) flag[i] = c.pinv[i] >= 0;
  __syncthreads();
  float4 a[NR][PW / 2];   // rows tid + k T: (re, im) of columns 2h and 2h + 1
  c64 n[NR];              // their column t
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int i = tid + k * T;
    const float4* src = reinterpret_cast<const float4*>(P + (size_t)(i < B ? i : 0) * LD);
#pragma unroll
    for (int h = 0; h < PW / 2; ++h) a[k][h] = src[h];
    n[k] = mk<float>(a[k][0].x, a[k][0].y);
  }
  unsigned best = 0;
#pragma unroll
  for (int k = 0; k < NR; ++k)
    if (!fl[k]) best = max(best, pivot_key32(cabs2(n[k]), tid + k * T));
  for (int i = tid + NR * T; i < B; i += T)
    if (!flag[i]) best = max(best, pivot_key32(cabs2(P[i * LD]), i));
  c64* Ccol = c.C + (size_t)slot * B;   // colmods of the panel's slots
#pragma unroll 1
  for (int t = 0; t < nbp; ++t) {
    best = __reduce_max_sync(0xffffffffu, best);
    if (lane == 0) wkey[warp] = best;
    __syncthreads();
    const unsigned kb = __reduce_max_sync(0xffffffffu, lane < NW ? wkey[lane] : 0u);
    const int r = min(2047 - (int)(kb & 2047u), B - 1);
    if (r % T == tid) {   // this thread holds the pivot row
      const int kr = r / T;
      float4* pr = reinterpret_cast<float4*>(P + (size_t)r * LD);
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (kr == k) {
#pragma unroll
          for (int h = 0; h < PW / 2; ++h) pr[h] = a[k][h];
          fl[k] = true;
        }
      if (kr >= NR) flag[r] = 1;
      const c64 inv = cinv(P[(size_t)r * LD + t]);
      float4* rv = reinterpret_cast<float4*>(rho);
#pragma unroll 1
      for (int h = 0; h < PW / 2; ++h) {
        const float4 x = pr[h];
        const c64 x0 = 2 * h == t ? inv + mk<float>(1, 0) : mk<float>(x.x, x.y) * inv;
        const c64 x1 = 2 * h + 1 == t ? inv + mk<float>(1, 0) : mk<float>(x.z, x.w) * inv;
        rv[h] = make_float4(x0.re, x0.im, x1.re, x1.im);
      }
      spiv[t] = r;
      sinv[t] = inv;
    }
    __syncthreads();
    const float4* rv = reinterpret_cast<const float4*>(rho);
    c64 ci[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int i = tid + k * T;
      ci[k] = n[k];
      if (i == r) ci[k].re -= 1.f;
      if (i < B) Ccol[(size_t)t * B + i] = ci[k];
    }
    const int hn = (t + 1) >> 1;
    const bool odd = (t + 1) & 1;
#pragma unroll
    for (int h = 0; h < PW / 2; ++h) {   // all register rows; rho read once
      const float4 b = rv[h];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        a[k][h].x = fmaf(-ci[k].re, b.x, fmaf(ci[k].im, b.y, a[k][h].x));
        a[k][h].y = fmaf(-ci[k].re, b.y, fmaf(-ci[k].im, b.x, a[k][h].y));
        a[k][h].z = fmaf(-ci[k].re, b.z, fmaf(ci[k].im, b.w, a[k][h].z));
        a[k][h].w = fmaf(-ci[k].re, b.w, fmaf(-ci[k].im, b.z, a[k][h].w));
        if (h == hn) n[k] = odd ? mk<float>(a[k][h].z, a[k][h].w) : mk<float>(a[k][h].x, a[k][h].y);
      }
    }
    best = 0;
    if (t + 1 < nbp) {
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (!fl[k]) best = max(best, pivot_key32(cabs2(n[k]), tid + k * T));
    }
    for (int i = tid + NR * T; i < B; i += T) {
      c64* row = P + (size_t)i * LD;
      c64 cs = row[t];
      if (i == r) cs.re -= 1.f;
      Ccol[(size_t)t * B + i] = cs;
      panel_row_update<float, PW, LD>(row, rho, cs);
      // the vector stores above and the element load below touch the same
      // words: keep the compiler from reordering them
      asm volatile("" ::: "memory");
      if (t + 1 < nbp && !flag[i]) best = max(best, pivot_key32(cabs2(row[t + 1]), i));
    }
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int i = tid + k * T;
    if (i < B) {
      float4* d = reinterpret_cast<float4*>(P + (size_t)i * LD);
#pragma unroll
      for (int h = 0; h < PW / 2; ++h) d[h] = a[k][h];
    }
  }
  __syncthreads();
  if (tid < nbp) {
    const int r = spiv[tid];
    c.piv[p0 + tid] = r;
    c.pinv[r] = p0 + tid;
    c.prow[slot + tid] = r;
    c.pinfo[slot + tid] = sinv[tid];
  }
  for (int e = tid; e < B * PW; e += T) {
    const int i = e / PW, q = e - i * PW;
    if (q < nbp) c.S[(size_t)i * B + p0 + q] = P[i * LD + q];
  }
}

// Pivot rows' other columns for the panel [p0, p0 + nbp), slots slot ..
// slot + nbp of the outer block [P0, P0 + kb) (one thread per column j
// outside the panel).  Columns inside the outer block are kept current by the
// inner updates:
//   rho_t[j] = (S[r_t][j] - sum_{s<t} C[r_t][s] rho_s[j]) / S[r_t][p0+t]   (s, t in the panel);
// columns outside it have not been updated since the block began, so the
// earlier slots of the block enter as well (delayed update):
//   rho_t[j] = (S[r_t][j] - sum_{s<slot} C[r_t][s] rho_s[j] - sum_{panel s<t} ...) / S[r_t][p0+t].
// Zero on the panel columns (the panel kernel has finished them).  Dynamic
// shared memory: Cp [NB][NB] (in-panel colmods at the pivot rows) and Cq
// [NB][slot] (earlier slots).
template <typename R, int PW>
__global__ void __launch_bounds__(128, sizeof(R) * PW <= 64 ? 7 : 1) gj_rowmod_kernel(const FChain<R>* chains, int p0, int P0,
                                                         int KBw) {
  pdl_wait3();
  // 32 columns per CTA; warp w takes a quarter of the earlier slots of the
  // delayed sum, warp 0 adds the quarters and runs the in-panel recurrence
  const FChain<R> c = chains[blockIdx.y];
  const int B = c.B;
  if (p0 >= B) return;
  const int nbp = min(PW, B - p0), slot = p0 - P0, blk_hi = min(P0 + KBw, B);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Cp = (cplx<R>*)smem_raw;              // [PW][PW]
  cplx<R>* Cq = Cp + PW * PW;                    // [PW][slot]
  cplx<R>* part = Cq + PW * slot;                // [3][PW][32]
  __shared__ cplx<R> inv[PW];
  __shared__ int pr[PW];
  for (int t = threadIdx.x; t < PW; t += blockDim.x) {
    inv[t] = t < nbp ? c.pinfo[slot + t] : mk<R>(0, 0);
    pr[t] = t < nbp ? c.prow[slot + t] : 0;
  }
  __syncthreads();
  // the colmods at the pivot rows: scattered single elements, all of a
  // thread's copies in flight at once (cp.async)
  for (int e = threadIdx.x; e < PW * PW; e += blockDim.x) {
    const int t = e / PW, q = e - t * PW;
    if (t < nbp && q < t)
      cp_async_el3(Cp + e, c.C + (size_t)(slot + q) * B + pr[t]);
    else
      Cp[e] = mk<R>(0, 0);
  }
  for (int e = threadIdx.x; e < PW * slot; e += blockDim.x) {
    const int t = e / slot, q = e - t * slot;
    if (t < nbp)
      cp_async_el3(Cq + e, c.C + (size_t)q * B + pr[t]);
    else
      Cq[e] = mk<R>(0, 0);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int j = blockIdx.x * 32 + lane;
  const bool live = j < B && (j < p0 || j >= p0 + nbp);
  const bool outside = j < P0 || j >= blk_hi;
  cplx<R> a[PW];
#pragma unroll
  for (int t = 0; t < PW; ++t) a[t] = mk<R>(0, 0);
  if (live && outside) {                          // this warp's quarter of the delayed sum
    const int qn = (slot + 3) / 4, q0 = warp * qn, q1 = min(slot, q0 + qn);
    constexpr int kUnroll = sizeof(cplx<R>) * PW <= 128 ? 8 : 4;   // loads in flight, within registers
#pragma unroll kUnroll
    for (int q = q0; q < q1; ++q) {
      const cplx<R> x = c.Rm[(size_t)q * B + j];
#pragma unroll
      for (int t = 0; t < PW; ++t) a[t] = a[t] - Cq[t * slot + q] * x;
    }
  }
  if (warp > 0) {
#pragma unroll
    for (int t = 0; t < PW; ++t) part[((warp - 1) * PW + t) * 32 + lane] = a[t];
  }
  __syncthreads();
  if (warp > 0 || j >= B) return;
  if (!live) {                                    // panel column: the panel kernel finished it
    for (int t = 0; t < nbp; ++t) c.Rm[(size_t)(slot + t) * B + j] = mk<R>(0, 0);
    return;
  }
#pragma unroll
  for (int t = 0; t < PW; ++t) {
    cplx<R> v = t < nbp ? c.S[(size_t)pr[t] * B + j] : mk<R>(0, 0);
    if (outside)
      v = v + a[t] + part[(0 * PW + t) * 32 + lane] + part[(1 * PW + t) * 32 + lane] +
          part[(2 * PW + t) * 32 + lane];
    a[t] = v;
  }
#pragma unroll
  for (int t = 0; t < PW; ++t) {
    if (t < nbp) {
      // two partial sums: half the dependent FMA chain of the recurrence
      cplx<R> s0 = a[t], s1 = mk<R>(0, 0);
#pragma unroll
      for (int q = 0; q + 1 < t; q += 2) {
        s0 = s0 - Cp[t * PW + q] * a[q];
        s1 = s1 - Cp[t * PW + q + 1] * a[q + 1];
      }
      if (t & 1) s0 = s0 - Cp[t * PW + t - 1] * a[t - 1];
      a[t] = (s0 + s1) * inv[t];
      c.Rm[(size_t)(slot + t) * B + j] = a[t];
    }
  }
}

template <typename R>
size_t rowmod_smem(int pw, int slot) {
  return (size_t)pw * (pw + slot + 3 * 32) * sizeof(cplx<R>);
}

// S[i][j] -= sum_{t < depth} C[slot + t][i] Rm[slot + t][j], 64 x 64 tile per
// CTA (256 threads, 4 x 4 outputs each: rows ty + 16 a, columns tx + 16 b),
// depth in chunks of NB through shared memory.  inner: the panel [base,
// base + depth) of the outer block [P0, P0 + KBw) updates the block's other
// columns (slots from base - P0); else the outer block's colmods and rowmods
// (slots 0 .. depth) update every column outside the block.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1) gj_update_kernel(const FChain<R>* chains, int base,
                                                        int width, int P0, int KBw, int inner) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.z];
  const int B = c.B;
  if (base >= B) return;
  const int depth = min(width, B - base), slot = base - P0;
  int wlo, whi, xlo, xhi;
  if (inner) {
    wlo = P0; whi = min(P0 + KBw, B); xlo = base; xhi = base + depth;
  } else {
    wlo = 0; whi = B; xlo = P0; xhi = min(P0 + KBw, B);
  }
  const int i0 = blockIdx.y * 64, j0 = wlo + blockIdx.x * 64;
  if (i0 >= B || j0 >= whi) return;
  if (j0 >= xlo && j0 + 64 <= xhi) return;       // excluded columns only: nothing to do
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Cs = (cplx<R>*)smem_raw;              // [64][NB + 1]
  cplx<R>* Rs = Cs + 64 * (NB + 1);              // [NB][64]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cplx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<R>(0, 0);
  for (int k0 = 0; k0 < depth; k0 += NB) {
    const int tmax = min(NB, depth - k0);         // a 16-column panel fills half a chunk
    // colmods [slot][B], rowmods [slot][B]: the chunk's tmax rows, all of a
    // thread's copies in flight at once (cp.async)
    for (int e = threadIdx.x; e < 64 * tmax; e += 256) {
      const int t = e / 64, q = e - t * 64;
      const size_t row = (size_t)(slot + k0 + t) * B;
      if (i0 + q < B)
        cp_async_el3(Cs + q * (NB + 1) + t, c.C + row + i0 + q);
      else
        Cs[q * (NB + 1) + t] = mk<R>(0, 0);
      if (j0 + q < whi)
        cp_async_el3(Rs + t * 64 + q, c.Rm + row + j0 + q);
      else
        Rs[t * 64 + q] = mk<R>(0, 0);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < tmax; ++t) {
      cplx<R> cv[4], rv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) cv[a] = Cs[(ty + 16 * a) * (NB + 1) + t];
#pragma unroll
      for (int b = 0; b < 4; ++b) rv[b] = Rs[t * 64 + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], cv[a], rv[b]);
    }
    __syncthreads();
  }
  // all sixteen loads before the stores (in flight together)
  cplx<R> sv[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      const bool ok = i < B && j < whi && (j < xlo || j >= xhi);
      sv[a][b] = ok ? c.S[(size_t)i * B + j] : mk<R>(0, 0);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= B) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j >= whi || (j >= xlo && j < xhi)) continue;
      c.S[(size_t)i * B + j] = sv[a][b] - acc[a][b];
    }
  }
}

// G_k[p][col] = S[piv[p]][pinv[col]] (undo the implicit pivoting).
template <typename R>
__global__ void __launch_bounds__(256) gj_writeout_kernel(const FChain<R>* chains) {
  pdl_wait3();
  const FChain<R> c = chains[blockIdx.z];
  const int col = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (col >= c.B || p >= c.B) return;
  const cplx<R> v = c.S[(size_t)c.piv[p] * c.B + c.pinv[col]];
  c.G[(size_t)c.k * c.bstride + (size_t)p * c.B + col] = v;
  if (c.Gp) {   // the same entry as tensor-core operand: row tile p / 128, depth chunk col / 16
    const int nkc = (c.B + 15) / 16;
    float* t = c.Gp + (size_t)c.k * c.gp_layer + ((size_t)(p >> 7) * nkc + (col >> 4)) * 8192 +
               tc::kmajor_off(p & 127, col & 15, 4) / 4;
    float hi, lo;
    tc::split_tf32((float)v.re, hi, lo);
    t[0] = hi;
    t[2048] = lo;
    tc::split_tf32((float)v.im, hi, lo);
    t[4096] = hi;
    t[6144] = lo;
  }
}

size_t update_smem(size_t el) { return (64 * (NB + 1) + NB * 64) * el; }

// The outer-block update of the complex64 factorisation on the tensor cores
// (tcgen05, kind::tf32, FP32 accumulation in tensor memory):
//   S[i][j] -= sum_{t < kb} C[t][i] Rm[t][j]   (j outside [P0, P0 + kb)).
// Complex products as real ones, Dr = Cr Rr - Ci Ri and Di = Cr Ri + Ci Rr,
// each real product in three TF32 passes (x = hi + lo: hi hi + hi lo + lo hi)
// so that the result keeps about FP32 accuracy.
//
// tc_pack_kernel splits the block's colmods and rowmods once into TF32 hi /
// lo planes laid out as the MMA operands: per 128-row tile (rows of S for C,
// columns of S for Rm) and per stage of kTcK depth, four K-major 128 x kTcK
// tiles (re hi, re lo, im hi, im lo), 32 KB contiguous; rowmods of the
// block's own columns and depths >= kb are zero.  gj_update_tc_kernel then
// takes one 128 x 128 tile of S per CTA: warp 0 streams the stages (one 32 KB
// bulk copy of each operand per stage, kTcBuf buffers), warp 1 issues the
// stage's 24 MMAs (128 x 128 x 8) once its copies have landed and commits
// them to the buffer's release barrier; Dr and Di accumulate in tensor-memory
// columns [0, 128) and [128, 256).  The epilogue moves them through shared
// memory (rows XOR-swizzled) and subtracts them from S in coalesced rows.
// Every wait is bounded (device flag on timeout).
constexpr int kTcM = 128;          // tile rows (MMA M) and columns (MMA N)
constexpr int kTcK = 16;           // complex depth per stage
constexpr int kTcBuf = 3;          // stage buffers
constexpr uint32_t kTcTile = kTcM * kTcK * 4;    // one TF32 operand tile: 8 KB
constexpr uint32_t kTcHalf = 4 * kTcTile;        // one operand's stage: re hi/lo, im hi/lo
constexpr uint32_t kTcStage = 2 * kTcHalf;       // C half then Rm half: 64 KB
constexpr size_t kTcSmem = kTcBuf * (size_t)kTcStage + 128;
// packed operand floats per chain and operand: row tiles x stages (KO / kTcK) x 32 KB
size_t tc_pack_floats(int Bmax, int KO) {
  return (size_t)((Bmax + kTcM - 1) / kTcM) * (KO / kTcK) * (kTcHalf / 4);
}

// grid (row tiles, stages, 2 x chains): z even packs C (rows i), odd Rm
// (columns j); thread r takes row r of the tile, four depths per 16-byte store.
__global__ void __launch_bounds__(128) tc_pack_kernel(const FChain<float>* chains, int P0, int KBw) {
  pdl_wait3();
  const FChain<float> c = chains[blockIdx.z >> 1];
  const bool isC = (blockIdx.z & 1) == 0;
  const int B = c.B;
  if (P0 >= B) return;
  const int kb = min(KBw, B - P0), xhi = P0 + kb;
  const int tile = blockIdx.x, st = blockIdx.y, r = threadIdx.x;
  const int q = tile * kTcM + r;                  // row i of S (C) or column j (Rm)
  float* out = (isC ? c.Ap : c.Bp) + ((size_t)tile * (KBw / kTcK) + st) * (kTcHalf / 4);
  const c64* src = isC ? c.C : c.Rm;
  const bool live = q < B && (isC || q < P0 || q >= xhi);
#pragma unroll
  for (int kg = 0; kg < kTcK; kg += 4) {
    float4 v[4];
    float* f = (float*)v;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = st * kTcK + kg + u;
      const c64 x = (live && kk < kb) ? src[(size_t)kk * B + q] : mk<float>(0, 0);
      tc::split_tf32(x.re, f[0 * 4 + u], f[1 * 4 + u]);
      tc::split_tf32(x.im, f[2 * 4 + u], f[3 * 4 + u]);
    }
    const uint32_t off = tc::kmajor_off(r, kg, kTcK / 4) / 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) *(float4*)(out + t * (kTcTile / 4) + off) = v[t];
  }
}

__global__ void __launch_bounds__(128, 1) gj_update_tc_kernel(const FChain<float>* chains, int P0,
                                                              int KBw, int* flag) {
  pdl_wait3();
  const FChain<float> c = chains[blockIdx.z];
  const int B = c.B;
  if (P0 >= B) return;
  const int kb = min(KBw, B - P0), xlo = P0, xhi = P0 + kb;
  const int i0 = blockIdx.y * kTcM, j0 = blockIdx.x * kTcM;
  if (i0 >= B || j0 >= B) return;
  if (j0 >= xlo && j0 + kTcM <= xhi) return;     // excluded columns only
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* full = (uint64_t*)(sm + kTcBuf * kTcStage);   // [kTcBuf] operands landed
  uint64_t* empty = full + kTcBuf;                          // [kTcBuf] buffer released
  uint64_t* done = empty + kTcBuf;                          // all MMAs complete
  uint32_t* tptr = (uint32_t*)(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < kTcBuf; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tptr, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tptr;
  const int nst = (kb + kTcK - 1) / kTcK;
  bool ok = true;
  if (warp == 0 && lane == 0) {                   // producer: bulk copies of the packed operands
    const float* Ap = c.Ap + (size_t)blockIdx.y * (KBw / kTcK) * (kTcHalf / 4);
    const float* Bp = c.Bp + (size_t)blockIdx.x * (KBw / kTcK) * (kTcHalf / 4);
    for (int st = 0; st < nst && ok; ++st) {
      const int buf = st % kTcBuf;
      if (st >= kTcBuf) ok = mbar_wait(&empty[buf], ((st - kTcBuf) / kTcBuf) & 1, flag);
      if (!ok) break;
      unsigned char* dst = sm + buf * kTcStage;
      mbar_expect_tx(&full[buf], kTcStage);
      tma_load_1d(dst, Ap + (size_t)st * (kTcHalf / 4), kTcHalf, &full[buf]);
      tma_load_1d(dst + kTcHalf, Bp + (size_t)st * (kTcHalf / 4), kTcHalf, &full[buf]);
    }
  } else if (warp == 1 && lane == 0) {            // MMA issuer
    constexpr uint32_t lbo = 128, sbo = (kTcK / 4) * 128;
    constexpr uint32_t id = tc::idesc_tf32(kTcM, kTcM, false);
    constexpr uint32_t idn = tc::idesc_tf32(kTcM, kTcM, true);
    for (int st = 0; st < nst && ok; ++st) {
      const int buf = st % kTcBuf;
      ok = mbar_wait(&full[buf], (st / kTcBuf) & 1, flag);
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t sb = smem_u32(sm + buf * kTcStage);
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint32_t ko = ks * 256;             // two core matrices along K per MMA
        auto d = [&](int t) { return tc::smem_desc(sb + t * kTcTile + ko, lbo, sbo); };
        const bool acc = st > 0 || ks > 0;
        // tiles: 0 Cr hi, 1 Cr lo, 2 Ci hi, 3 Ci lo, 4 Rr hi, 5 Rr lo, 6 Ri hi, 7 Ri lo
        tc::mma_tf32(tmem, d(0), d(4), id, acc);          // Dr += Cr Rr
        tc::mma_tf32(tmem, d(0), d(5), id, true);
        tc::mma_tf32(tmem, d(1), d(4), id, true);
        tc::mma_tf32(tmem, d(2), d(6), idn, true);        // Dr -= Ci Ri
        tc::mma_tf32(tmem, d(2), d(7), idn, true);
        tc::mma_tf32(tmem, d(3), d(6), idn, true);
        tc::mma_tf32(tmem + 128, d(0), d(6), id, acc);    // Di += Cr Ri
        tc::mma_tf32(tmem + 128, d(0), d(7), id, true);
        tc::mma_tf32(tmem + 128, d(1), d(6), id, true);
        tc::mma_tf32(tmem + 128, d(2), d(4), id, true);   // Di += Ci Rr
        tc::mma_tf32(tmem + 128, d(2), d(5), id, true);
        tc::mma_tf32(tmem + 128, d(3), d(4), id, true);
      }
      tc::commit(&empty[buf]);
    }
    if (ok) tc::commit(done);                     // covers every MMA issued before it
  }
  __syncwarp();
  ok = mbar_wait(done, 0, flag);
  ok = __syncthreads_and(ok);
  tc::fence_after_sync();
  c64* D = (c64*)sm;                              // [128][128], column XOR-swizzled by row
  const int row = warp * 32 + lane;
  if (ok) {
#pragma unroll 1
    for (int cc = 0; cc < kTcM; cc += 32) {
      float vr[32], vi[32];
      tc::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + cc, vr);
      tc::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + 128 + cc, vi);
#pragma unroll
      for (int q = 0; q < 32; ++q) D[row * kTcM + ((cc + q) ^ (row & 31))] = mk<float>(vr[q], vi[q]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (ok) {
    // thread: columns j0 + cp, j0 + cp + 1 of the rows 2 u + rs; sixteen rows'
    // loads are issued before any store, so that they are in flight together
    const int cp = (tid & 63) * 2, rs = tid >> 6;
    const int j = j0 + cp;
    const bool c0 = j < B && (j < xlo || j >= xhi);
    const bool c1 = j + 1 < B && (j + 1 < xlo || j + 1 >= xhi);
#pragma unroll 1
    for (int rb = 0; rb < kTcM; rb += 32) {
      float2 x0[16], x1[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int i = i0 + rb + 2 * u + rs;
        const float2* p = (const float2*)(c.S + (size_t)i * B + j);
        x0[u] = (i < B && c0) ? p[0] : make_float2(0.f, 0.f);
        x1[u] = (i < B && c1) ? p[1] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int rr = rb + 2 * u + rs, i = i0 + rr;
        if (i >= B) continue;
        float2* p = (float2*)(c.S + (size_t)i * B + j);
        const int sw = rr & 31;
        if (c0) {
          const c64 v = D[rr * kTcM + (cp ^ sw)];
          p[0] = make_float2(x0[u].x - v.re, x0[u].y - v.im);
        }
        if (c1) {
          const c64 v = D[rr * kTcM + ((cp + 1) ^ sw)];
          p[1] = make_float2(x1[u].x - v.re, x1[u].y - v.im);
        }
      }
    }
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 256);
  }
}

// ------------------------------------------------------------------- solves
// Right-hand side of a 3-D slab solve (SubdomSolve, Table 2) into the layer
// fields Y[k][r][b] (rhs r of the chunk, layer stride ldl): a raw slab field
// [nr][N_t][W] (N_t = nz ny), or the gather of the global columns (ga, gb] of
// f [nr][nz][ny][nx] plus the injections of Eqs. 19-20 at the local columns
// ef, ef+1 (from B1) and eb, eb+1 (from B3), transmission buffers
// [2][nr_tot][N_t] (rhs r0 + r).
template <typename R>
struct Rhs3 {
  const cplx<R>* raw;
  const cplx<R>* f;
  int nx, lo, wl, ga, gb;
  const cplx<R>* B1;
  int ef;
  const cplx<R>* B3;
  int eb;
  const cplx<R>* inj;        // [4][N_t][9]
  int r0, nr_tot;
};

template <typename R>
__global__ void slab3_rhs_kernel(Rhs3<R> q, int W, int ny, int nz, cplx<R>* Y, size_t ldl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y, r = blockIdx.z;
  const int B = W * ny;
  if (b >= B) return;
  const int y = b / W, e = b - y * W;
  const size_t nt = (size_t)ny * nz;
  const int rr = q.r0 + r;
  cplx<R> v = mk<R>(0, 0);
  if (q.raw) {
    v = q.raw[((size_t)r * nz + k) * B + b];
  } else {
    const int g = e - q.wl + q.lo;
    if (g > q.ga && g <= q.gb) v = q.f[(((size_t)r * nz + k) * ny + y) * q.nx + g];
    auto inject = [&](int s, const cplx<R>* Bf) {   // s: 0..3 (coefficient set)
      const cplx<R>* c = q.inj + ((size_t)s * nt + (size_t)k * ny + y) * 9;
      const cplx<R>* Bl = Bf + ((size_t)(1 - (s & 1)) * q.nr_tot + rr) * nt;
      for (int t = 0; t < 9; ++t) {
        const int kk = k + t / 3 - 1, yy = y + t % 3 - 1;
        if (kk >= 0 && kk < nz && yy >= 0 && yy < ny) cfma(v, c[t], Bl[(size_t)kk * ny + yy]);
      }
    };
    if (q.ef >= 0 && e == q.ef) inject(0, q.B1);        // row beta uses B[1]
    if (q.ef >= 0 && e == q.ef + 1) inject(1, q.B1);    // row beta+1 uses B[0]
    if (q.eb >= 0 && e == q.eb) inject(2, q.B3);
    if (q.eb >= 0 && e == q.eb + 1) inject(3, q.B3);
  }
  Y[(size_t)k * ldl + (size_t)r * B + b] = v;
}

// One coupling term applied to a layer field: sum over (dy, dx) of
// st[k][q(dz, dy, dx)][b] X[r][b + dy W + dx] (only (0, 0) for the 7-point
// operator).
template <typename R>
struct Cpl3 {
  int k, dz;
  const cplx<R>* X;          // [nr][B]
};
template <typename R>
struct Piece3 {
  const cplx<R>* base;       // [nr][B] or null
  cplx<R>* out;              // [nr][B]
  int nc;
  Cpl3<R> c[2];
};
template <typename R>
struct Prep3 {
  int B, W, ny, nr, diag;
  R sgn;                     // out = base + sgn * (sum of the couplings)
  const cplx<R>* st;
  int np;
  Piece3<R> p[2];
  // complex64 tensor-core products with at most 32 right-hand sides: out is
  // written straight into the packed operand (TF32 hi/lo planes, the layout
  // tc_vpack_kernel writes) instead, nkc chunks per piece; null otherwise
  float* vp;
  int nkc;
};

template <typename R>
__global__ void slab3_prep_kernel(Prep3<R> a) {
  pdl_wait3();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const Piece3<R>& P = a.p[blockIdx.z];
  if (b >= a.B) return;
  const int y = b / a.W, e = b - y * a.W;
  cplx<R> acc = mk<R>(0, 0);
  for (int c = 0; c < P.nc; ++c) {
    const cplx<R>* st = a.st + (size_t)P.c[c].k * 27 * a.B;
    const cplx<R>* X = P.c[c].X + (size_t)r * a.B;
    const int dz = P.c[c].dz;
    if (a.diag) {
      cfma(acc, st[(size_t)qidx(dz, 0, 0) * a.B + b], X[b]);
    } else {
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= a.ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int ee = e + dx;
          if (ee < 0 || ee >= a.W) continue;
          cfma(acc, st[(size_t)qidx(dz, dy, dx) * a.B + b], X[yy * a.W + ee]);
        }
      }
    }
  }
  const size_t o = (size_t)r * a.B + b;
  cplx<R> v = P.base ? P.base[o] : mk<R>(0, 0);
  v.re += a.sgn * acc.re;
  v.im += a.sgn * acc.im;
  if constexpr (std::is_same<R, float>::value) {
    if (a.vp) {   // planes re hi, re lo, im hi, im lo of chunk b / 16, row r, k = b mod 16
      float* q = a.vp + ((size_t)blockIdx.z * a.nkc + (b >> 4)) * 2048 + tc::kmajor_off(r, b & 15, 4) / 4;
      float hi, lo;
      tc::split_tf32(v.re, hi, lo);
      q[0] = hi;
      q[512] = lo;
      tc::split_tf32(v.im, hi, lo);
      q[1024] = hi;
      q[1536] = lo;
      return;
    }
  }
  P.out[o] = v;
}

// Dense layer GEMV with the stored inverse, up to two pieces (the two
// chains): y[r][i] = G[i][:] v[r][:] (mode 0) or y[r][i] - G[i][:] v[r][:]
// (mode 1), r < NR.
constexpr int kGemvRows = 4;
// The coupling term of a chain's next layer step, computed by the reduction
// of the current step (diagonal couplings, complex64 tensor-core path, one
// chunk of right-hand sides): V' = base' + sgn * st' x, with x the layer just
// solved, written packed into piece slot z of the next step.
template <typename R>
struct NextPiece {
  const cplx<R>* st;         // [B] the next layer's coupling plane, null: no next step
  const cplx<R>* base;       // [nr][B] or null
  int z;
};
template <typename R>
struct NextCpl {
  float* vp;                 // packed operand of the next step, null: not fused
  int nkc;
  R sgn;
  NextPiece<R> p[2];
};

template <typename R>
struct GemvPiece {
  const cplx<R>* G;          // [B][B]
  const cplx<R>* v;          // [nr][B]
  cplx<R>* y;                // [nr][B]
};
template <typename R>
struct Gemv3 {
  int B, nr, mode, np;
  GemvPiece<R> p[2];
};

// A CTA takes kGemvRows rows; its 8 warps split the columns into 8 chunks
// (many independent loads in flight per SM), each lane accumulates the
// products of its columns, and the partial sums are reduced across lanes
// (shuffles) and across the warps (shared memory).
template <typename R, int NR>
__global__ void __launch_bounds__(256) slab3_gemv_kernel(Gemv3<R> a) {
  pdl_wait3();
  const GemvPiece<R> P = blockIdx.y == 0 ? a.p[0] : a.p[1];   // static parameter offsets
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = a.B;
  const int i0 = blockIdx.x * kGemvRows;
  if (i0 >= B) return;
  const int cw = (B + 7) / 8;
  const int j0 = warp * cw, j1 = min(B, j0 + cw);
  __shared__ cplx<R> part[8][kGemvRows * NR];
  // right-hand sides in chunks of NR (the CTA's rows of G stay in cache)
  for (int r0 = 0; r0 < a.nr; r0 += NR) {
  const int nrc = min(NR, a.nr - r0);
  cplx<R> acc[kGemvRows][NR];
#pragma unroll
  for (int q = 0; q < kGemvRows; ++q)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[q][r] = mk<R>(0, 0);
  for (int j = j0 + lane; j < j1; j += 32) {
    cplx<R> v[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = r < nrc ? P.v[(size_t)(r0 + r) * B + j] : mk<R>(0, 0);
#pragma unroll
    for (int q = 0; q < kGemvRows; ++q) {
      const int i = i0 + q;
      const cplx<R> g = i < B ? P.G[(size_t)i * B + j] : mk<R>(0, 0);
#pragma unroll
      for (int r = 0; r < NR; ++r) cfma(acc[q][r], g, v[r]);
    }
  }
#pragma unroll
  for (int q = 0; q < kGemvRows; ++q)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc[q][r].re += __shfl_xor_sync(0xffffffffu, acc[q][r].re, o);
        acc[q][r].im += __shfl_xor_sync(0xffffffffu, acc[q][r].im, o);
      }
      if (lane == 0) part[warp][q * NR + r] = acc[q][r];
    }
  __syncthreads();
  if (threadIdx.x < kGemvRows * NR) {
    const int q = threadIdx.x / NR, r = threadIdx.x - q * NR;
    const int i = i0 + q;
    if (i < B && r < nrc) {
      cplx<R> s = mk<R>(0, 0);
#pragma unroll
      for (int w = 0; w < 8; ++w) s = s + part[w][threadIdx.x];
      cplx<R>* out = P.y + (size_t)(r0 + r) * B + i;
      *out = a.mode == 0 ? s : *out - s;
    }
  }
  __syncthreads();            // part is reused by the next chunk
  }
}

// The layer product for many right-hand sides as a register-tiled complex
// GEMM, Y (B x nr) = G (B x B) V (B x nr): a CTA takes 128 rows x 32
// right-hand sides over one of `nsplit` column ranges (split K, so that
// about four CTAs run per SM), streams G and V through shared memory in
// depth chunks of GK, and each thread accumulates 4 rows (ty + 32 q) x 4
// right-hand sides.  The partial sums go to part [np][nsplit][nr][B]; the
// reduce kernel adds them in a fixed order (deterministic) into y.
constexpr int kG3Rows = 128, kG3Rhs = 32;
template <typename R> struct G3K { static constexpr int v = 32; };
template <> struct G3K<double> { static constexpr int v = 16; };

template <typename R>
__global__ void __launch_bounds__(256) slab3_gemm_kernel(Gemv3<R> a, int nsplit, cplx<R>* part) {
  pdl_wait3();
  constexpr int GK = G3K<R>::v;
  const GemvPiece<R> P = blockIdx.z == 0 ? a.p[0] : a.p[1];
  const int B = a.B, tid = threadIdx.x;
  const int i0 = blockIdx.x * kG3Rows, sp = blockIdx.y;
  const int kper = (B + nsplit - 1) / nsplit;
  const int klo = sp * kper, khi = min(B, klo + kper);
  __shared__ cplx<R> Gs[kG3Rows][GK + 1];
  __shared__ cplx<R> Vs[kG3Rhs][GK + 1];
  const int tx = tid & 7, ty = tid >> 3;          // rhs 4 tx .. 4 tx + 3, rows ty + 32 q
  cplx<R>* pout = part + ((size_t)blockIdx.z * nsplit + sp) * a.nr * B;
  for (int r0 = 0; r0 < a.nr; r0 += kG3Rhs) {
    cplx<R> acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q][u] = mk<R>(0, 0);
    for (int k0 = klo; k0 < khi; k0 += GK) {
      for (int e = tid; e < kG3Rows * GK; e += 256) {
        const int rr = e / GK, k = e - rr * GK;
        const int i = i0 + rr, kk = k0 + k;
        Gs[rr][k] = (i < B && kk < khi) ? P.G[(size_t)i * B + kk] : mk<R>(0, 0);
      }
      for (int e = tid; e < kG3Rhs * GK; e += 256) {
        const int r = e / GK, k = e - r * GK;
        const int kk = k0 + k;
        Vs[r][k] = (r0 + r < a.nr && kk < khi) ? P.v[(size_t)(r0 + r) * B + kk] : mk<R>(0, 0);
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < GK; ++k) {
        cplx<R> g[4], v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) g[q] = Gs[ty + 32 * q][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = Vs[4 * tx + u][k];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) cfma(acc[q][u], g[q], v[u]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty + 32 * q;
      if (i >= B) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + 4 * tx + u;
        if (r < a.nr) pout[(size_t)r * B + i] = acc[q][u];
      }
    }
  }
}

template <typename R>
__global__ void slab3_gemm_reduce_kernel(Gemv3<R> a, int nsplit, const cplx<R>* part,
                                         NextCpl<R> nx) {
  pdl_wait3();
  const GemvPiece<R> P = blockIdx.z == 0 ? a.p[0] : a.p[1];
  const int B = a.B;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (i >= B || r >= a.nr) return;
  const cplx<R>* pp = part + (size_t)blockIdx.z * nsplit * a.nr * B + (size_t)r * B + i;
  cplx<R> s = mk<R>(0, 0);
  for (int sp = 0; sp < nsplit; ++sp) s = s + pp[(size_t)sp * a.nr * B];
  cplx<R>* out = P.y + (size_t)r * B + i;
  const cplx<R> x = a.mode == 0 ? s : *out - s;
  *out = x;
  if constexpr (std::is_same<R, float>::value) {
    // the next layer's right-hand side of this chain, written packed: the
    // same arithmetic as slab3_prep_kernel with one diagonal coupling
    const NextPiece<R> N = blockIdx.z == 0 ? nx.p[0] : nx.p[1];   // static parameter offsets
    if (nx.vp && N.st) {
      cplx<R> acc = mk<R>(0, 0);
      cfma(acc, N.st[i], x);
      cplx<R> v = N.base ? N.base[(size_t)r * B + i] : mk<R>(0, 0);
      v.re += nx.sgn * acc.re;
      v.im += nx.sgn * acc.im;
      float* q = nx.vp + ((size_t)N.z * nx.nkc + (i >> 4)) * 2048 + tc::kmajor_off(r, i & 15, 4) / 4;
      float hi, lo;
      tc::split_tf32(v.re, hi, lo);
      q[0] = hi;
      q[512] = lo;
      tc::split_tf32(v.im, hi, lo);
      q[1024] = hi;
      q[1536] = lo;
    }
  }
}

// The layer product on the tensor cores (complex64, more than four right-
// hand sides): Y (B x nr) = G V with G packed at write-out (row tiles of
// 128, depth chunks of 16, four TF32 planes re hi / lo, im hi / lo) and V
// packed per call by tc_vpack_kernel (N = 32 right-hand-side rows per chunk).
// One CTA per row tile and K range (split K): warp 0 streams the chunks (a
// 32 KB and an 8 KB bulk copy per stage), warp 1 issues the chunk's 24 MMAs
// (M = 128, N = 32, K = 8; three TF32 passes per real product) into Dr / Di
// (tensor-memory columns [0, 32) and [32, 64)), and the four warps write
// the row tile's partial sums to part [np][nsplit][nr][B] (reduced by
// slab3_gemm_reduce_kernel).  Right-hand sides in chunks of 32 (one pass of
// the K range per chunk).  Every wait is bounded.
constexpr int kTgN = 32;                                // right-hand sides per MMA (N)
constexpr uint32_t kTgA = 4 * 8192;                     // G chunk: 4 planes x 128 x 16 TF32
constexpr uint32_t kTgB = 4 * 2048;                     // V chunk: 4 planes x 32 x 16 TF32
constexpr uint32_t kTgStage = kTgA + kTgB;              // 40 KB
constexpr int kTgBuf = 4;
constexpr size_t kTgSmem = kTgBuf * (size_t)kTgStage + 128;

// V [nr][B] (rows r0 .. r0 + 31) -> Vp [nkc][4 planes][32 x 16] K-major (2 KB per
// plane); one thread per (rhs row, depth chunk), four depths per 16-byte store
__global__ void __launch_bounds__(128) tc_vpack_kernel(Gemv3<float> a, int r0, float* vp_all) {
  pdl_wait3();
  const GemvPiece<float> P = blockIdx.z == 0 ? a.p[0] : a.p[1];
  const int B = a.B, nkc = (B + 15) / 16;
  float* vp = vp_all + (size_t)blockIdx.z * nkc * 2048;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = e & 31, kc = e >> 5;
  if (kc >= nkc) return;
  const int rr = r0 + r;
#pragma unroll
  for (int kg = 0; kg < 16; kg += 4) {
    float4 v[4];
    float* f = (float*)v;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = kc * 16 + kg + u;
      const c64 x = (rr < a.nr && j < B) ? P.v[(size_t)rr * B + j] : mk<float>(0, 0);
      tc::split_tf32(x.re, f[0 * 4 + u], f[1 * 4 + u]);
      tc::split_tf32(x.im, f[2 * 4 + u], f[3 * 4 + u]);
    }
    float* out = vp + (size_t)kc * 2048 + tc::kmajor_off(r, kg, 4) / 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) *(float4*)(out + t * 512) = v[t];
  }
}

__global__ void __launch_bounds__(128, 1) slab3_gemm_tc_kernel(Gemv3<float> a, const float* gp0,
                                                               const float* gp1, int nsplit,
                                                               const float* vp_all, int r0,
                                                               c64* part, int* flag) {
  pdl_wait3();
  const int B = a.B, nkc = (B + 15) / 16, rt = blockIdx.x, sp = blockIdx.y, pc = blockIdx.z;
  const int kper = (nkc + nsplit - 1) / nsplit;
  const int kc0 = sp * kper, kc1 = min(nkc, kc0 + kper);
  const int nst = kc1 - kc0;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* full = (uint64_t*)(sm + kTgBuf * kTgStage);
  uint64_t* empty = full + kTgBuf;
  uint64_t* done = empty + kTgBuf;
  uint32_t* tptr = (uint32_t*)(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < kTgBuf; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tptr, 64);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tptr;
  bool ok = true;
  if (nst > 0) {
    if (warp == 0 && lane == 0) {               // producer
      const float* G = (pc == 0 ? gp0 : gp1) + (size_t)rt * nkc * 8192;
      const float* V = vp_all + (size_t)pc * nkc * 2048;
      for (int st = 0; st < nst && ok; ++st) {
        const int buf = st % kTgBuf;
        if (st >= kTgBuf) ok = mbar_wait(&empty[buf], ((st - kTgBuf) / kTgBuf) & 1, flag);
        if (!ok) break;
        unsigned char* dst = sm + buf * kTgStage;
        mbar_expect_tx(&full[buf], kTgStage);
        tma_load_1d(dst, G + (size_t)(kc0 + st) * 8192, kTgA, &full[buf]);
        tma_load_1d(dst + kTgA, V + (size_t)(kc0 + st) * 2048, kTgB, &full[buf]);
      }
    } else if (warp == 1 && lane == 0) {        // MMA issuer
      constexpr uint32_t lbo = 128, sbo = 4 * 128;
      constexpr uint32_t id = tc::idesc_tf32(128, kTgN, false);
      constexpr uint32_t idn = tc::idesc_tf32(128, kTgN, true);
      for (int st = 0; st < nst && ok; ++st) {
        const int buf = st % kTgBuf;
        ok = mbar_wait(&full[buf], (st / kTgBuf) & 1, flag);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t sa = smem_u32(sm + buf * kTgStage), sbb = sa + kTgA;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ko = ks * 256;
          auto A = [&](int t) { return tc::smem_desc(sa + t * 8192 + ko, lbo, sbo); };
          auto Bd = [&](int t) { return tc::smem_desc(sbb + t * 2048 + ko, lbo, sbo); };
          const bool acc = st > 0 || ks > 0;
          // planes: 0 re hi, 1 re lo, 2 im hi, 3 im lo (G: A, V: B)
          tc::mma_tf32(tmem, A(0), Bd(0), id, acc);          // Dr += Gr Vr
          tc::mma_tf32(tmem, A(0), Bd(1), id, true);
          tc::mma_tf32(tmem, A(1), Bd(0), id, true);
          tc::mma_tf32(tmem, A(2), Bd(2), idn, true);        // Dr -= Gi Vi
          tc::mma_tf32(tmem, A(2), Bd(3), idn, true);
          tc::mma_tf32(tmem, A(3), Bd(2), idn, true);
          tc::mma_tf32(tmem + 32, A(0), Bd(2), id, acc);     // Di += Gr Vi
          tc::mma_tf32(tmem + 32, A(0), Bd(3), id, true);
          tc::mma_tf32(tmem + 32, A(1), Bd(2), id, true);
          tc::mma_tf32(tmem + 32, A(2), Bd(0), id, true);    // Di += Gi Vr
          tc::mma_tf32(tmem + 32, A(2), Bd(1), id, true);
          tc::mma_tf32(tmem + 32, A(3), Bd(0), id, true);
        }
        tc::commit(&empty[buf]);
      }
      if (ok) tc::commit(done);
    }
    __syncwarp();
    ok = mbar_wait(done, 0, flag);
  }
  ok = __syncthreads_and(ok);
  tc::fence_after_sync();
  const int i = rt * 128 + warp * 32 + lane;
  if (ok) {
    float vr[32], vi[32];
    if (nst > 0) {
      tc::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16), vr);
      tc::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + 32, vi);
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) vr[q] = vi[q] = 0.f;
    }
    if (i < B) {
      c64* po = part + ((size_t)pc * nsplit + sp) * a.nr * B;
#pragma unroll
      for (int q = 0; q < 32; ++q)
        if (r0 + q < a.nr) po[(size_t)(r0 + q) * B + i] = mk<float>(vr[q], vi[q]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 64);
  }
}

// Epilogue of a 3-D slab solve (Table 2): the slab solution's core columns
// (ua, ub] into the global field, the layers at e2, e2+1 (B2) and e4, e4+1
// (B4) for the transmission, or the whole slab field (raw).
template <typename R>
struct Out3 {
  cplx<R>* raw;              // [nr][N_t][W]
  cplx<R>* u;                // [nr][nz][ny][nx]
  int nx, lo, wl, ua, ub;
  cplx<R>* B2;
  int e2;
  cplx<R>* B4;
  int e4;
  int r0, nr_tot;
};

template <typename R>
__global__ void slab3_out_kernel(Out3<R> o, int W, int ny, int nz, const cplx<R>* Y, size_t ldl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y, r = blockIdx.z;
  const int B = W * ny;
  if (b >= B) return;
  const int y = b / W, e = b - y * W;
  const size_t nt = (size_t)ny * nz;
  const int rr = o.r0 + r;
  const cplx<R> v = Y[(size_t)k * ldl + (size_t)r * B + b];
  if (o.raw) {
    o.raw[((size_t)r * nz + k) * B + b] = v;
    return;
  }
  const int g = e - o.wl + o.lo;
  if (g > o.ua && g <= o.ub) o.u[(((size_t)r * nz + k) * ny + y) * o.nx + g] = v;
  const size_t idx = (size_t)k * ny + y;
  if (o.B2 && (e == o.e2 || e == o.e2 + 1))
    o.B2[((size_t)(e - o.e2) * o.nr_tot + rr) * nt + idx] = v;
  if (o.B4 && (e == o.e4 || e == o.e4 + 1))
    o.B4[((size_t)(e - o.e4) * o.nr_tot + rr) * nt + idx] = v;
}

}  // namespace

// ---------------------------------------------------------------- host side
// Chains: 2 (j - 1) = top chain of slab j (layers 0 .. m-1), 2 (j - 1) + 1 =
// bottom chain (layers nz-1 .. m+1); step t factors layer t of the top and
// nz-1-t of the bottom chains; the meeting step factors layer m of every
// slab (with the top chain's work buffers).
template <typename R>
void factor_level3d(hz_handle* h, Level& L, cudaStream_t s) {
  const int J = L.J, nz = L.nz, m = L.mid;
  const int ntop = m, nbot = nz - 1 - m, T = std::max(ntop, nbot);
  const size_t el = sizeof(cplx<R>);
  int Bmax = 0;
  for (int j = 1; j <= J; ++j) Bmax = std::max(Bmax, L.slabs[j].B);
  const int nch = 2 * J;
  // outer block width (a multiple of both panel widths)
  const int KO = h->p.block_3d > 0 ? h->p.block_3d : kOuterDefault;
  const size_t sS = (size_t)Bmax * Bmax, sC = (size_t)Bmax * KO;
  if (!L.f3_S) {   // work buffers and descriptors: built by the first factorisation, kept
    L.f3_S = dmalloc(el * sS * nch);
    L.f3_C = dmalloc(el * sC * nch);
    L.f3_R = dmalloc(el * sC * nch + el * KO * nch);
    L.f3_piv = (int*)dmalloc(sizeof(int) * ((size_t)2 * Bmax + KO) * nch);
    const size_t npk = tc_pack_floats(Bmax, KO);
    if (sizeof(R) == 4) L.f3_pack = (float*)dmalloc(sizeof(float) * npk * 2 * nch);
    std::vector<FChain<R>> all;
    auto chain = [&](int j, int c) {
      const Slab& S = L.slabs[j];
      FChain<R> f{};
      f.B = S.B; f.W = S.W; f.ny = L.ny;
      f.st = (const cplx<R>*)S.st3;
      f.G = (cplx<R>*)S.G;
      f.bstride = S.bstride;
      f.Gp = S.Gp;
      f.gp_layer = S.gp_layer;
      f.S = (cplx<R>*)L.f3_S + sS * c;
      f.C = (cplx<R>*)L.f3_C + sC * c;
      f.Rm = (cplx<R>*)L.f3_R + sC * c;
      f.pinfo = (cplx<R>*)L.f3_R + sC * nch + (size_t)KO * c;
      int* ip = L.f3_piv + ((size_t)2 * Bmax + KO) * c;
      f.piv = ip; f.pinv = ip + Bmax; f.prow = ip + 2 * Bmax;
      if (L.f3_pack) {
        f.Ap = L.f3_pack + npk * 2 * c;
        f.Bp = f.Ap + npk;
      }
      return f;
    };
    for (int t = 0; t < T; ++t)
      for (int j = 1; j <= J; ++j) {
        if (t < ntop) {
          FChain<R> f = chain(j, 2 * (j - 1));
          f.k = t; f.nterm = t > 0 ? 1 : 0;
          f.kp[0] = t - 1; f.dzL[0] = -1; f.dzR[0] = +1;
          all.push_back(f);
        }
        if (t < nbot) {
          FChain<R> f = chain(j, 2 * (j - 1) + 1);
          f.k = nz - 1 - t; f.nterm = t > 0 ? 1 : 0;
          f.kp[0] = nz - t; f.dzL[0] = +1; f.dzR[0] = -1;
          all.push_back(f);
        }
      }
    for (int j = 1; j <= J; ++j) {
      FChain<R> f = chain(j, 2 * (j - 1));
      f.k = m; f.nterm = 2;
      f.kp[0] = m - 1; f.dzL[0] = -1; f.dzR[0] = +1;
      f.kp[1] = m + 1; f.dzL[1] = +1; f.dzR[1] = -1;
      all.push_back(f);
    }
    L.f3_desc = dmalloc(sizeof(FChain<R>) * all.size());
    HZ_CU(cudaMemcpyAsync(L.f3_desc, all.data(), sizeof(FChain<R>) * all.size(),
                          cudaMemcpyHostToDevice, s));
    HZ_CU(cudaFuncSetAttribute(gj_update_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)update_smem(el)));
    HZ_CU(cudaFuncSetAttribute(gj_rowmod_kernel<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rowmod_smem<R>(16, kOuterMax)));
    HZ_CU(cudaFuncSetAttribute(gj_rowmod_kernel<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rowmod_smem<R>(NB, kOuterMax)));
    HZ_CU(cudaFuncSetAttribute(gj_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTcSmem));
  }
  const FChain<R>* desc = (const FChain<R>*)L.f3_desc;
  const int fe = L.fe ? 1 : 0;
  // complex64 outer updates on the tensor cores (HZ_TEST_NO_TC=1: the FP32
  // SIMT kernel instead, for comparison)
  const bool use_tc = sizeof(R) == 4 && test_hook("HZ_TEST_NO_TC") <= 0;
  // panels of 16 columns held in shared memory when a block's panel fits
  // (complex64 rows padded to 18 elements for vector access where those fit,
  // else to 17), else panels of NB columns eliminated in place in global memory
  // (complex64 with 18-element rows: the register-resident form)
  constexpr bool c64_path = std::is_same<R, float>::value;
  const size_t psm_v = c64_path ? panel_reg_smem_bytes<16>(Bmax) : panel_smem_bytes<R, 16, 17>(Bmax);
  const size_t psm_o = panel_smem_bytes<R, 16, 17>(Bmax);
  const size_t smem_cap = (size_t)225 * 1024;
  const bool smem_panel = Bmax < 2047 && psm_o <= smem_cap;   // 11-bit row field of the pivot keys
  const bool vec_panel = smem_panel && psm_v <= smem_cap;
  const size_t psm = vec_panel ? psm_v : psm_o;
  void (*panel_fn)(const FChain<R>*, int, int) = gj_panel_smem_kernel<R, 16, 17>;
  int panel_threads = kSmemPanelThreads;
  if constexpr (c64_path) {
    if (vec_panel) {   // all rows in registers up to 1344 (448 threads x 3), else 1024 of them
      const bool three = Bmax > 1024 && Bmax <= 448 * 3;
      panel_fn = three ? gj_panel_reg_kernel<16, 448, 3> : gj_panel_reg_kernel<16, 512, 2>;
      panel_threads = three ? 448 : 512;
    }
  }
  const int nbw = smem_panel ? 16 : NB;
  if (smem_panel)
    HZ_CU(cudaFuncSetAttribute(panel_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
  auto layer = [&](const FChain<R>* d, int cnt, int nterm) {
    const dim3 gs(cdiv(Bmax, 128), Bmax, cnt);
    timed(h, "slab_factor3d_schur", 0.0, s, [&] {
      if (!fe) {
        launch_pdl3(schur_S_kernel<R>, gs, 128, s, d, -1, 1, 0);
      } else {
        launch_pdl3(schur_S_kernel<R>, gs, 128, s, d, -1, 1, 1);
        for (int t = 0; t < nterm; ++t) {
          launch_pdl3(schur_T_kernel<R>, gs, 128, s, d, t);
          launch_pdl3(schur_S_kernel<R>, gs, 128, s, d, t, 0, 1);
        }
      }
    });
    h->launches += fe ? 1 + 2 * nterm : 1;
    // outer blocks of KO columns: inner panels of nbw columns update the
    // block's own columns (rank nbw); the block's colmods and rowmods then
    // update every other column at once (rank KO; tensor cores in complex64)
    for (int P0 = 0; P0 < Bmax; P0 += KO) {
      const int bw = std::min(KO, Bmax - P0);
      for (int p0 = P0; p0 < P0 + bw; p0 += nbw) {
        const int slot = p0 - P0;
        timed(h, "slab_factor3d_panel", 0.0, s, [&] {
          if (smem_panel)
            launch_pdl3s(panel_fn, dim3(cnt), panel_threads, psm, s, d, p0, slot);
          else
            launch_pdl3(gj_panel_kernel<R>, dim3(cnt), kPanelThreads, s, d, p0, slot);
        });
        timed(h, "slab_factor3d_rowmod", 0.0, s, [&] {
          if (nbw == 16)
            launch_pdl3s(gj_rowmod_kernel<R, 16>, dim3(cdiv(Bmax, 32), cnt), 128,
                         rowmod_smem<R>(16, slot), s, d, p0, P0, KO);
          else
            launch_pdl3s(gj_rowmod_kernel<R, NB>, dim3(cdiv(Bmax, 32), cnt), 128,
                         rowmod_smem<R>(NB, slot), s, d, p0, P0, KO);
        });
        const int nbp = std::min(nbw, Bmax - p0);
        const double fli = 8.0 * (double)Bmax * std::max(0, bw - nbp) * nbp * cnt;
        timed(h, "slab_factor3d_inner", fli, s, [&] {
          launch_pdl3s(gj_update_kernel<R>, dim3(cdiv(bw, 64), cdiv(Bmax, 64), cnt), 256,
                       update_smem(el), s, d, p0, nbw, P0, KO, 1);
        });
        h->launches += 3;
      }
      // algorithmic flop of the outer update: 8 B (B - kb) kb per chain (complex MACs x 8)
      const double fl = 8.0 * (double)Bmax * (Bmax - bw) * bw * cnt;
      if (Bmax > bw) {
        timed(h, "slab_factor3d_update", fl, s, [&] {
          if (use_tc) {
            launch_pdl3(tc_pack_kernel, dim3(cdiv(Bmax, kTcM), KO / kTcK, 2 * cnt), 128, s,
                        (const FChain<float>*)d, P0, KO);
            launch_pdl3s(gj_update_tc_kernel, dim3(cdiv(Bmax, kTcM), cdiv(Bmax, kTcM), cnt), 128,
                         kTcSmem, s, (const FChain<float>*)d, P0, KO, h->dev_flag);
          }
          else
            launch_pdl3s(gj_update_kernel<R>, dim3(cdiv(Bmax, 64), cdiv(Bmax, 64), cnt), 256,
                         update_smem(el), s, d, P0, KO, P0, KO, 0);
        });
        h->launches += use_tc ? 2 : 1;
      }
    }
    timed(h, "slab_factor3d_writeout", 0.0, s,
          [&] { launch_pdl3(gj_writeout_kernel<R>, dim3(cdiv(Bmax, 256), Bmax, cnt), 256, s, d); });
    h->launches += 1;
    HZ_CU(cudaGetLastError());
  };
  size_t off = 0;
  for (int t = 0; t < T; ++t) {
    const int cnt = J * ((t < ntop ? 1 : 0) + (t < nbot ? 1 : 0));
    layer(desc + off, cnt, t > 0 ? 1 : 0);
    off += cnt;
  }
  layer(desc + off, J, 2);
  HZ_CU(cudaStreamSynchronize(s));
  check_dev_flag(h, s);          // a bounded tensor-core wait that gave up
}

namespace {

// One 3-D slab solve for right-hand sides [r0, r0 + nr) of nr_tot: rhs
// gather, forward chains, meeting layer, backward chains, epilogue.
template <typename R, int NR>
void run_solve3d(hz_handle* h, Level& L, Slab& S, Rhs3<R> q, Out3<R> o, int nr, cudaStream_t s) {
  const int B = S.B, nz = L.nz, m = L.mid;
  const int ntop = m, nbot = nz - 1 - m, T = std::max(ntop, nbot);
  const size_t ldl = (size_t)nr * B;      // layer stride of the chunk's Y
  cplx<R>* Y = (cplx<R>*)S.Y;
  cplx<R>* V = (cplx<R>*)S.V;
  cplx<R>* V1 = V + (size_t)nr * B;
  const cplx<R>* G = (const cplx<R>*)S.G;
  auto Yk = [&](int k) { return Y + (size_t)k * ldl; };
  auto Gk = [&](int k) { return G + (size_t)k * S.bstride; };
  const double el = sizeof(cplx<R>);
  const double gbytes = (double)B * B * el;
  slab3_rhs_kernel<R><<<dim3(cdiv(B, 128), nz, nr), 128, 0, s>>>(q, S.W, L.ny, nz, Y, ldl);
  Prep3<R> pa{};
  pa.B = B; pa.W = S.W; pa.ny = L.ny; pa.nr = nr; pa.diag = L.fe ? 0 : 1;
  pa.st = (const cplx<R>*)S.st3;
  Gemv3<R> ga{};
  ga.B = B; ga.nr = nr;
  const unsigned gblocks = (unsigned)cdiv(B, kGemvRows);
  auto prep = [&](int np) {
    pa.np = np;
    launch_pdl3(slab3_prep_kernel<R>, dim3(cdiv(B, 128), nr, np), 128, s, pa);
    h->launches++;
  };
  // many right-hand sides: the split-K register-tiled GEMM and its reduction
  // (partial sums in the slab's GEMM scratch); few: the GEMV kernel
  const bool tiled = nr > 4 && S.gpart != nullptr;
  // complex64: the tensor-core product with the packed inverses
  const bool tcg = tiled && S.Gp != nullptr && test_hook("HZ_TEST_NO_TC") <= 0;
  static bool tg_attr = false;
  if (tcg && !tg_attr) {
    HZ_CU(cudaFuncSetAttribute(slab3_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTgSmem));
    tg_attr = true;
  }
  const int nkc = cdiv(B, 16), nrt = cdiv(B, 128);
  // one chunk of right-hand sides: the coupling kernel packs the operand
  // itself (no tc_vpack_kernel launch per layer)
  const bool fuse_pack = tcg && nr <= kTgN;
  if (fuse_pack) {
    pa.vp = S.Vp;
    pa.nkc = nkc;
  }
  // K splits of the tensor-core products: one wave of CTAs (one per SM), so
  // that no second, nearly empty wave follows
  auto nsplit_of = [&](int np) {
    return std::max(1, std::min(kG3MaxSplit, h->sms / (np * nrt)));
  };
  auto gp_of = [&](const cplx<R>* Gl) {   // packed inverse of the layer whose G is Gl
    const size_t layer = (size_t)(Gl - G) / S.bstride;
    return S.Gp + layer * S.gp_layer;
  };
  const int nI = cdiv(B, kG3Rows);
  // at least ~4 CTAs per SM (two pieces), so that the last wave is short
  const int nsplit = std::max(1, std::min(kG3MaxSplit, cdiv(4 * h->sms, 2 * nI)));
  // complex64 tensor-core path with diagonal couplings: the reduction of a
  // layer step also forms the next step's packed right-hand side, so that
  // slab3_prep_kernel runs only for the first step of each sweep and the
  // meeting layer.  next_of(t, fwd): the next step's coupling per piece.
  const bool fuse_next = fuse_pack && pa.diag;
  auto next_of = [&](int t, bool fwd) {
    NextCpl<R> nx{};
    if (!fuse_next || t + 1 >= T) return nx;
    nx.vp = S.Vp;
    nx.nkc = nkc;
    nx.sgn = fwd ? (R)-1 : (R)1;
    int z = 0, zn = 0;
    for (int side = 0; side < 2; ++side) {
      const int len = side == 0 ? ntop : nbot;
      if (t >= len) continue;                 // this side has no step t
      NextPiece<R>& N = nx.p[z++];
      if (t + 1 >= len) continue;             // nor a step t + 1 (N.st stays null)
      const int k = fwd ? (side == 0 ? t : nz - 1 - t) : (side == 0 ? m - 1 - t : m + 1 + t);
      const int kn = side == 0 ? (fwd ? k + 1 : k - 1) : (fwd ? k - 1 : k + 1);
      const int dz = (side == 0) == fwd ? -1 : +1;
      N.st = pa.st + ((size_t)kn * 27 + qidx(dz, 0, 0)) * B;
      N.base = fwd ? Yk(kn) : nullptr;
      N.z = zn++;
    }
    return nx;
  };
  auto gemv = [&](int np, int mode, const NextCpl<R>& nx) {
    ga.np = np;
    ga.mode = mode;
    timed(h, "slab3_gemv", np * (gbytes + 2.0 * nr * B * el), s, [&] {
      if (tcg) {
        if constexpr (std::is_same<R, float>::value) {
          c64* part = (c64*)S.gpart;
          const float* g0 = gp_of(ga.p[0].G);
          const float* g1 = np > 1 ? gp_of(ga.p[1].G) : g0;
          const int nsplit_tc = nsplit_of(np);
          for (int r0 = 0; r0 < nr; r0 += kTgN) {
            if (!fuse_pack) {
              launch_pdl3(tc_vpack_kernel, dim3(cdiv(32 * nkc, 128), 1, np), 128, s, ga, r0, S.Vp);
              h->launches++;
            }
            launch_pdl3s(slab3_gemm_tc_kernel, dim3(nrt, nsplit_tc, np), 128, kTgSmem, s, ga, g0,
                         g1, nsplit_tc, (const float*)S.Vp, r0, part, h->dev_flag);
            h->launches++;
          }
          launch_pdl3(slab3_gemm_reduce_kernel<float>, dim3(cdiv(B, 128), nr, np), 128, s, ga,
                      nsplit_tc, (const c64*)part, nx);
        }
      } else if (tiled) {
        cplx<R>* part = (cplx<R>*)S.gpart;
        launch_pdl3(slab3_gemm_kernel<R>, dim3(nI, nsplit, np), 256, s, ga, nsplit, part);
        launch_pdl3(slab3_gemm_reduce_kernel<R>, dim3(cdiv(B, 128), nr, np), 128, s, ga, nsplit,
                    (const cplx<R>*)part, NextCpl<R>{});
        h->launches++;
      } else {
        launch_pdl3(slab3_gemv_kernel<R, NR>, dim3(gblocks, np), 256, s, ga);
      }
    });
  };
  // forward: y_t = G_t (f_t - L_t y_{t-1}), both chains per launch
  bool packed = false;   // this step's packed right-hand side written by the last reduction
  for (int t = 0; t < T; ++t) {
    int np = 0;
    for (int side = 0; side < 2; ++side) {
      if (t >= (side == 0 ? ntop : nbot)) continue;
      const int k = side == 0 ? t : nz - 1 - t;
      const int kp = side == 0 ? k - 1 : k + 1;
      cplx<R>* Vp = np == 0 ? V : V1;
      pa.p[np].base = Yk(k);
      pa.p[np].out = Vp;
      pa.p[np].nc = t > 0 ? 1 : 0;
      pa.p[np].c[0] = Cpl3<R>{k, side == 0 ? -1 : +1, Yk(kp)};
      ga.p[np] = GemvPiece<R>{Gk(k), Vp, Yk(k)};
      ++np;
    }
    pa.sgn = (R)-1;
    if (!packed) prep(np);
    const NextCpl<R> nx = next_of(t, true);
    gemv(np, 0, nx);
    packed = nx.vp != nullptr;
  }
  // meeting: x_m = G_m (f_m - C_m y_{m-1} - B_m y_{m+1})
  pa.p[0].base = Yk(m);
  pa.p[0].out = V;
  pa.p[0].nc = 2;
  pa.p[0].c[0] = Cpl3<R>{m, -1, Yk(m - 1)};
  pa.p[0].c[1] = Cpl3<R>{m, +1, Yk(m + 1)};
  pa.sgn = (R)-1;
  prep(1);
  ga.p[0] = GemvPiece<R>{Gk(m), V, Yk(m)};
  gemv(1, 0, NextCpl<R>{});
  packed = false;
  // backward: x_t = y_t - G_t R_t x_{t+1}, outwards from the meeting layer
  for (int t = 0; t < T; ++t) {
    int np = 0;
    for (int side = 0; side < 2; ++side) {
      if (t >= (side == 0 ? ntop : nbot)) continue;
      const int k = side == 0 ? m - 1 - t : m + 1 + t;
      const int kn = side == 0 ? k + 1 : k - 1;   // the next layer (towards m), solved
      cplx<R>* Vp = np == 0 ? V : V1;
      pa.p[np].base = nullptr;
      pa.p[np].out = Vp;
      pa.p[np].nc = 1;
      pa.p[np].c[0] = Cpl3<R>{k, side == 0 ? +1 : -1, Yk(kn)};
      ga.p[np] = GemvPiece<R>{Gk(k), Vp, Yk(k)};
      ++np;
    }
    pa.sgn = (R)1;
    if (!packed) prep(np);
    const NextCpl<R> nx = next_of(t, false);
    gemv(np, 1, nx);
    packed = nx.vp != nullptr;
  }
  slab3_out_kernel<R><<<dim3(cdiv(B, 128), nz, nr), 128, 0, s>>>(o, S.W, L.ny, nz, Y, ldl);
  h->launches += 2 + (2 * T + 1);   // rhs and out kernels, one reduction or GEMV per step
  HZ_CU(cudaGetLastError());
}

// All right-hand sides in one pass; the GEMV takes them in chunks of at most
// 8 (its compile-time accumulators) inside each launch.
template <typename R>
void run_solve3d_all(hz_handle* h, Level& L, Slab& S, Rhs3<R> q, Out3<R> o, int n_rhs,
                     cudaStream_t s) {
  q.nr_tot = o.nr_tot = n_rhs;
  q.r0 = o.r0 = 0;
  if (n_rhs == 1) run_solve3d<R, 1>(h, L, S, q, o, n_rhs, s);
  else if (n_rhs == 2) run_solve3d<R, 2>(h, L, S, q, o, n_rhs, s);
  else if (n_rhs <= 4) run_solve3d<R, 4>(h, L, S, q, o, n_rhs, s);
  else run_solve3d<R, 8>(h, L, S, q, o, n_rhs, s);
}

}  // namespace

template <typename R>
void subdom_solve3d(hz_handle* h, Level& L, int j, const cplx<R>* f, int a, int b, int at,
                    int bt, bool tau1, const cplx<R>* B1, bool tau2, cplx<R>* B2, bool tau3,
                    const cplx<R>* B3, bool tau4, cplx<R>* B4, cplx<R>* u, int n_rhs,
                    cudaStream_t s) {
  Slab& S = L.slabs[j];
  // transmission from or to a missing neighbour is dropped (T^(1) = T~^(J) = 0)
  tau1 = tau1 && j > 1;
  tau4 = tau4 && j > 1;
  tau2 = tau2 && j < L.J;
  tau3 = tau3 && j < L.J;
  auto loc = [&](int g) { return g - S.lo + S.wl; };
  Rhs3<R> q{};
  q.f = f; q.nx = L.nx; q.lo = S.lo; q.wl = S.wl; q.ga = a; q.gb = b;
  q.B1 = B1; q.ef = tau1 ? loc(L.beta[j - 1]) : -1;
  q.B3 = B3; q.eb = tau3 ? loc(L.beta_t[j]) : -1;
  q.inj = (const cplx<R>*)S.inj3;
  Out3<R> o{};
  o.u = u; o.nx = L.nx; o.lo = S.lo; o.wl = S.wl; o.ua = at; o.ub = bt;
  o.B2 = tau2 ? B2 : nullptr; o.e2 = tau2 ? loc(L.beta[j]) : -1;
  o.B4 = tau4 ? B4 : nullptr; o.e4 = tau4 ? loc(L.beta_t[j - 1]) : -1;
  timed(h, "slab_solve3d", 0.0, s, [&] { run_solve3d_all<R>(h, L, S, q, o, n_rhs, s); });
}

template <typename R>
void slab_solve_raw3d(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud, int n_rhs,
                      cudaStream_t s) {
  Slab& S = L.slabs[j];
  Rhs3<R> q{};
  q.raw = fd; q.ef = -1; q.eb = -1;
  Out3<R> o{};
  o.raw = ud; o.e2 = -1; o.e4 = -1;
  run_solve3d_all<R>(h, L, S, q, o, n_rhs, s);
}

template void build_slabs3d<float>(hz_handle*, Level&, cudaStream_t);
template void build_slabs3d<double>(hz_handle*, Level&, cudaStream_t);
template void factor_level3d<float>(hz_handle*, Level&, cudaStream_t);
template void factor_level3d<double>(hz_handle*, Level&, cudaStream_t);
template void subdom_solve3d<float>(hz_handle*, Level&, int, const c64*, int, int, int, int, bool,
                                    const c64*, bool, c64*, bool, const c64*, bool, c64*, c64*,
                                    int, cudaStream_t);
template void subdom_solve3d<double>(hz_handle*, Level&, int, const c128*, int, int, int, int,
                                     bool, const c128*, bool, c128*, bool, const c128*, bool,
                                     c128*, c128*, int, cudaStream_t);
template void slab_solve_raw3d<float>(hz_handle*, Level&, int, const c64*, c64*, int,
                                      cudaStream_t);
template void slab_solve_raw3d<double>(hz_handle*, Level&, int, const c128*, c128*, int,
                                       cudaStream_t);

}  // namespace hz
