// Matrix-free Helmholtz operator kernels.
//
// Fine level: Eq. 40 multiplied by h^2, coefficients recomputed on the fly
// from m and the 1-D PML tables (1/alpha at unknowns, alpha at cell midpoints):
//   (A u)_{k,x} = (1/a2_k)(-a1_{x-1/2} u_{k,x-1} + (a1_{x-1/2}+a1_{x+1/2}) u_{k,x} - a1_{x+1/2} u_{k,x+1})
//               + (1/a1_x)(-a2_{k-1/2} u_{k-1,x} + (a2_{k-1/2}+a2_{k+1/2}) u_{k,x} - a2_{k+1/2} u_{k+1,x})
//               - h^2 omega^2 m_{k,x} / (a1_x a2_k) u_{k,x}
// with a_{i-1/2} = cell i and a_{i+1/2} = cell i+1, Dirichlet zeros outside.
// In the PML-free interior (alpha = 1 at the node and both adjacent cells
// along both axes) the coefficients are real and the row reduces to
//   (A u)_{k,x} = (4 - h^2 omega^2 m_{k,x}) u_{k,x} - u_{k,x-1} - u_{k,x+1} - u_{k-1,x} - u_{k+1,x},
// about a fifth of the general row's arithmetic (which matters most for the
// complex128 operator: GB300's FP64 pipe is narrow).
// Coarse level: a stored 9-point stencil (9 coefficient planes).
#include "hz_internal.h"

#include <utility>

namespace hz {

template <typename R> struct Tab;
template <> struct Tab<double> {
  static const c128* inode(const AxisTables& a) { return a.ia_node; }
  static const c128* cell(const AxisTables& a) { return a.a_cell; }
  static const double* beta(const AxisTables& a) { return a.beta; }
};
template <> struct Tab<float> {
  static const c64* inode(const AxisTables& a) { return a.ia_node32; }
  static const c64* cell(const AxisTables& a) { return a.a_cell32; }
  static const float* beta(const AxisTables& a) { return a.beta32; }
};
template <typename R> struct Med;
template <> struct Med<double> { static const double* m(const Level& L) { return L.m; } };
template <> struct Med<float> { static const float* m(const Level& L) { return L.m32; } };
template <typename R> struct Planes;
template <> struct Planes<double> { static const c128* st(const Level& L) { return L.st128; } };
template <> struct Planes<float> { static const c64* st(const Level& L) { return L.st64; } };

struct FdArgs {
  int nx, ny;
  double h2w2;
};

// Returns (A u)_{k,x} and the diagonal entry of A.
template <typename R>
__device__ __forceinline__ cplx<R> fd_row(const cplx<R>* __restrict__ u, int nx, int ny, int k,
                                          int x, R h2w2, const R* __restrict__ m,
                                          const cplx<R>* __restrict__ ia1n,
                                          const cplx<R>* __restrict__ a1c,
                                          const cplx<R>* __restrict__ ia2n,
                                          const cplx<R>* __restrict__ a2c, cplx<R>* diag,
                                          const R* __restrict__ bx = nullptr,
                                          const R* __restrict__ by = nullptr) {
  const cplx<R> z = mk<R>(0, 0);
  cplx<R> uc = u[(size_t)k * nx + x];
  cplx<R> ul = (x > 0) ? u[(size_t)k * nx + x - 1] : z;
  cplx<R> ur = (x < nx - 1) ? u[(size_t)k * nx + x + 1] : z;
  cplx<R> ud = (k > 0) ? u[(size_t)(k - 1) * nx + x] : z;
  cplx<R> uu = (k < ny - 1) ? u[(size_t)(k + 1) * nx + x] : z;
  cplx<R> ia2 = ia2n[k];
  cplx<R> ia1 = ia1n[x];
  cplx<R> l = a1c[x], r = a1c[x + 1], d = a2c[k], up = a2c[k + 1];
  cplx<R> tx = (l + r) * uc - l * ul - r * ur;
  cplx<R> ty = (d + up) * uc - d * ud - up * uu;
  cplx<R> mass = (h2w2 * m[(size_t)k * nx + x]) * (ia1 * ia2);
  if (bx) mass = mass * sponge_s<R>(bx[x] + by[k]);     // sponge: k^2 (1 + i beta)^2
  if (diag) *diag = ia2 * (l + r) + ia1 * (d + up) - mass;
  return ia2 * tx + ia1 * ty - mass * uc;
}

// Interior row (real coefficients); *diag = the real diagonal entry.
template <typename R>
__device__ __forceinline__ cplx<R> fd_row_interior(const cplx<R>* __restrict__ u, int nx, int ny,
                                                   int k, int x, R h2w2, const R* __restrict__ m,
                                                   R* diag) {
  const cplx<R> z = mk<R>(0, 0);
  const cplx<R> uc = u[(size_t)k * nx + x];
  const cplx<R> ul = (x > 0) ? u[(size_t)k * nx + x - 1] : z;
  const cplx<R> ur = (x < nx - 1) ? u[(size_t)k * nx + x + 1] : z;
  const cplx<R> ud = (k > 0) ? u[(size_t)(k - 1) * nx + x] : z;
  const cplx<R> uu = (k < ny - 1) ? u[(size_t)(k + 1) * nx + x] : z;
  const R c = (R)4 - h2w2 * m[(size_t)k * nx + x];
  *diag = c;
  return mk<R>(c * uc.re - ((ul.re + ur.re) + (ud.re + uu.re)),
               c * uc.im - ((ul.im + ur.im) + (ud.im + uu.im)));
}

template <typename R>
__device__ __forceinline__ cplx<R> st_row(const cplx<R>* __restrict__ u, int nx, int ny, int k,
                                          int x, const cplx<R>* __restrict__ st,
                                          cplx<R>* diag) {
  size_t plane = (size_t)nx * ny;
  cplx<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    int kk = k + dy;
    if (kk < 0 || kk >= ny) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      int xx = x + dx;
      if (xx < 0 || xx >= nx) continue;
      cfma(acc, st[(size_t)((dy + 1) * 3 + dx + 1) * plane + (size_t)k * nx + x],
           u[(size_t)kk * nx + xx]);
    }
  }
  if (diag) *diag = st[4 * plane + (size_t)k * nx + x];
  return acc;
}

// mode 0: y = A u;  mode 1: y = f - A u;
// mode 2 (Jacobi): y = u + omega (f - A u) / diag(A)
// (finite differences: rows x in [xlo, xhi], k in [ylo, yhi] take the
// interior form)
template <typename R, bool STORED>
__global__ void __launch_bounds__(256) op_kernel(int mode, int nx, int ny, R h2w2,
                                                 const R* __restrict__ m,
                                                 const cplx<R>* __restrict__ a1n,
                                                 const cplx<R>* __restrict__ a1c,
                                                 const cplx<R>* __restrict__ a2n,
                                                 const cplx<R>* __restrict__ a2c,
                                                 const cplx<R>* __restrict__ st,
                                                 const cplx<R>* __restrict__ f,
                                                 const cplx<R>* __restrict__ u,
                                                 cplx<R>* __restrict__ y, R omega_jac,
                                                 int xlo, int xhi, int ylo, int yhi,
                                                 const R* __restrict__ bx,
                                                 const R* __restrict__ by) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  int r = blockIdx.z;
  if (x >= nx) return;
  size_t off = (size_t)r * nx * ny;
  const cplx<R>* ur = u + off;
  size_t i = off + (size_t)k * nx + x;
  if (!STORED && x >= xlo && x <= xhi && k >= ylo && k <= yhi) {
    R dr;
    const cplx<R> au = fd_row_interior<R>(ur, nx, ny, k, x, h2w2, m, &dr);
    if (mode == 0) {
      y[i] = au;
    } else if (mode == 1) {
      y[i] = f[i] - au;
    } else {
      const R s = omega_jac / dr;
      const cplx<R> res = f[i] - au;
      const cplx<R> uc = ur[(size_t)k * nx + x];
      y[i] = mk<R>(uc.re + s * res.re, uc.im + s * res.im);
    }
    return;
  }
  cplx<R> dg;
  cplx<R> au = STORED ? st_row<R>(ur, nx, ny, k, x, st, mode == 2 ? &dg : nullptr)
                      : fd_row<R>(ur, nx, ny, k, x, h2w2, m, a1n, a1c, a2n, a2c,
                                  mode == 2 ? &dg : nullptr, bx, by);
  if (mode == 0) {
    y[i] = au;
  } else if (mode == 1) {
    y[i] = f[i] - au;
  } else {
    cplx<R> res = f[i] - au;
    y[i] = ur[(size_t)k * nx + x] + omega_jac * (res * cinv(dg));
  }
}

// Complex64 finite-difference rows, two consecutive unknowns e, e+1 of the
// flattened [y][x] field per thread: where both are interior points of one
// row (and the pair's addresses are 16-byte aligned) the centre values, the
// right-hand side and the result move as 128-bit accesses; elsewhere each
// point takes the rows above.  Same modes as op_kernel.
__global__ void __launch_bounds__(256) op_pair_kernel_c64(
    int mode, int nx, int ny, float h2w2, const float* __restrict__ m,
    const c64* __restrict__ a1n, const c64* __restrict__ a1c, const c64* __restrict__ a2n,
    const c64* __restrict__ a2c, const c64* __restrict__ f, const c64* __restrict__ u,
    c64* __restrict__ y, float omega_jac, int xlo, int xhi, int ylo, int yhi,
    const float* __restrict__ bx, const float* __restrict__ by) {
  const size_t n = (size_t)nx * ny;
  const size_t e = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (e >= n) return;
  const size_t off = (size_t)blockIdx.y * n;
  const c64* U = u + off;
  const int k = (int)(e / nx), x = (int)(e - (size_t)k * nx);
  const uintptr_t al = (uintptr_t)(U + e) | (uintptr_t)(y + off + e) |
                       (mode >= 1 ? (uintptr_t)(f + off + e) : (uintptr_t)0);
  const bool pair = e + 1 < n && x + 1 < nx && x >= xlo && x + 1 <= xhi && k >= ylo && k <= yhi &&
                    (al & 15) == 0;
  if (pair) {
    const float4 c = *reinterpret_cast<const float4*>(U + e);
    const c64 z = mk(0.f, 0.f);
    const c64 l = x > 0 ? U[e - 1] : z;
    const c64 r = x + 2 < nx ? U[e + 2] : z;
    const c64 d0 = k > 0 ? U[e - nx] : z, d1 = k > 0 ? U[e - nx + 1] : z;
    const c64 u0 = k < ny - 1 ? U[e + nx] : z, u1 = k < ny - 1 ? U[e + nx + 1] : z;
    const float2 mm = *reinterpret_cast<const float2*>(m + e);
    const float c0 = 4.f - h2w2 * mm.x, c1 = 4.f - h2w2 * mm.y;
    float4 a;
    a.x = c0 * c.x - ((l.re + c.z) + (d0.re + u0.re));
    a.y = c0 * c.y - ((l.im + c.w) + (d0.im + u0.im));
    a.z = c1 * c.z - ((c.x + r.re) + (d1.re + u1.re));
    a.w = c1 * c.w - ((c.y + r.im) + (d1.im + u1.im));
    float4 o;
    if (mode == 0) {
      o = a;
    } else {
      const float4 fv = *reinterpret_cast<const float4*>(f + off + e);
      if (mode == 1) {
        o = make_float4(fv.x - a.x, fv.y - a.y, fv.z - a.z, fv.w - a.w);
      } else {
        const float s0 = omega_jac / c0, s1 = omega_jac / c1;
        o = make_float4(c.x + s0 * (fv.x - a.x), c.y + s0 * (fv.y - a.y), c.z + s1 * (fv.z - a.z),
                        c.w + s1 * (fv.w - a.w));
      }
    }
    *reinterpret_cast<float4*>(y + off + e) = o;
    return;
  }
  for (size_t p = e; p < e + 2 && p < n; ++p) {
    const int kk = (int)(p / nx), xx = (int)(p - (size_t)kk * nx);
    const size_t i = off + p;
    c64 au;
    c64 dg = mk(0.f, 0.f);
    if (xx >= xlo && xx <= xhi && kk >= ylo && kk <= yhi) {
      float dr;
      au = fd_row_interior<float>(U, nx, ny, kk, xx, h2w2, m, &dr);
      dg = mk(dr, 0.f);
    } else {
      au = fd_row<float>(U, nx, ny, kk, xx, h2w2, m, a1n, a1c, a2n, a2c, mode == 2 ? &dg : nullptr,
                         bx, by);
    }
    if (mode == 0) y[i] = au;
    else if (mode == 1) y[i] = f[i] - au;
    else y[i] = U[p] + omega_jac * ((f[i] - au) * cinv(dg));
  }
}

template <typename R>
static void launch_op(hz_handle* h, const Level& L, int mode, const cplx<R>* f,
                      const cplx<R>* u, cplx<R>* y, int n_rhs, double omega_jac,
                      cudaStream_t s) {
  if (L.dim3d) {
    launch_op3d<R>(h, L, mode, f, u, y, n_rhs, omega_jac, s);
    return;
  }
  dim3 block(128);
  dim3 grid(cdiv(L.nx, 128), L.ny, n_rhs);
  R h2w2 = (R)(L.h * L.h * h->p.omega * h->p.omega);
  // algorithmic bytes: u read and y written once per dof, f once for modes 1 and
  // 2, and the medium (finite differences) or the 9 planes (stored stencil)
  const double el = sizeof(cplx<R>), dofs = (double)L.nx * L.ny * n_rhs;
  const double coef = L.fe ? 9.0 * el : (double)sizeof(R);
  const double bytes = dofs * (2.0 * el + (mode >= 1 ? el : 0.0) + coef);
  const char* tag = sizeof(R) == 4 ? "stencil_c64" : "stencil_c128";
  if (L.fe)
    timed(h, tag, bytes, s, [&] {
      op_kernel<R, true><<<grid, block, 0, s>>>(mode, L.nx, L.ny, h2w2, nullptr, nullptr, nullptr,
                                                nullptr, nullptr, Planes<R>::st(L), f, u, y,
                                                (R)omega_jac, 1, 0, 1, 0, nullptr, nullptr);
    });
  else if constexpr (sizeof(R) == 4)
    timed(h, tag, bytes, s, [&] {
      const size_t pairs = ((size_t)L.nx * L.ny + 1) / 2;
      op_pair_kernel_c64<<<dim3((unsigned)cdiv(pairs, 256), n_rhs), 256, 0, s>>>(
          mode, L.nx, L.ny, h2w2, Med<R>::m(L), Tab<R>::inode(L.ax), Tab<R>::cell(L.ax),
          Tab<R>::inode(L.ay), Tab<R>::cell(L.ay), f, u, y, (R)omega_jac, L.ax.in_lo, L.ax.in_hi,
          L.ay.in_lo, L.ay.in_hi, Tab<R>::beta(L.ax), Tab<R>::beta(L.ay));
    });
  else
    timed(h, tag, bytes, s, [&] {
      op_kernel<R, false><<<grid, block, 0, s>>>(
          mode, L.nx, L.ny, h2w2, Med<R>::m(L), Tab<R>::inode(L.ax), Tab<R>::cell(L.ax),
          Tab<R>::inode(L.ay), Tab<R>::cell(L.ay), nullptr, f, u, y, (R)omega_jac, L.ax.in_lo,
          L.ax.in_hi, L.ay.in_lo, L.ay.in_hi, Tab<R>::beta(L.ax), Tab<R>::beta(L.ay));
    });
  h->launches++;
  HZ_CU(cudaGetLastError());
}

template <typename R>
void level_apply(hz_handle* h, const Level& L, const cplx<R>* u, cplx<R>* y, int n_rhs,
                 cudaStream_t s) {
  launch_op<R>(h, L, 0, nullptr, u, y, n_rhs, 0.0, s);
}

template <typename R>
void level_residual(hz_handle* h, const Level& L, const cplx<R>* f, const cplx<R>* u,
                    cplx<R>* r, int n_rhs, cudaStream_t s) {
  launch_op<R>(h, L, 1, f, u, r, n_rhs, 0.0, s);
}

// nu omega-Jacobi steps u <- u + omega D^-1 (f - A u) (Section 4.1), ping-pong
// between u and t; the result ends in u (one copy when nu is odd).
template <typename R>
void jacobi_steps(hz_handle* h, const Level& L, const cplx<R>* f, cplx<R>* u, cplx<R>* t,
                  int nu, double omega_jac, int n_rhs, cudaStream_t s) {
  cplx<R>* a = u;
  cplx<R>* b = t;
  for (int i = 0; i < nu; ++i) {
    launch_op<R>(h, L, 2, f, a, b, n_rhs, omega_jac, s);
    std::swap(a, b);
  }
  if (a != u)
    HZ_CU(cudaMemcpyAsync(u, a, sizeof(cplx<R>) * (size_t)n_rhs * L.size(),
                          cudaMemcpyDeviceToDevice, s));
}

void apply_fine64(hz_handle* h, const c128* u, c128* y, int n_rhs, cudaStream_t s) {
  level_apply<double>(h, h->fine, u, y, n_rhs, s);
}

template <typename To, typename From>
__global__ void cast_kernel(const cplx<From>* a, cplx<To>* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = ccast<To>(a[i]);
}

template <typename To, typename From>
void cast_copy(const cplx<From>* a, cplx<To>* b, size_t n, cudaStream_t s) {
  cast_kernel<To, From><<<cdiv(n, 256), 256, 0, s>>>(a, b, n);
  HZ_CU(cudaGetLastError());
}

void check_dev_flag(hz_handle* h, cudaStream_t s) {
  int flag = 0;
  HZ_CU(cudaMemcpyAsync(&flag, h->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  HZ_CU(cudaStreamSynchronize(s));
  if (flag == DEV_TIMEOUT) {
    HZ_CU(cudaMemsetAsync(h->dev_flag, 0, sizeof(int), s));
    throw Failure(HZ_ETIMEOUT, "a bounded device-side wait gave up");
  }
  if (flag != DEV_OK) {
    HZ_CU(cudaMemsetAsync(h->dev_flag, 0, sizeof(int), s));
    throw Failure(HZ_ECUDA, "device error flag " + std::to_string(flag));
  }
}

template void level_apply<double>(hz_handle*, const Level&, const c128*, c128*, int, cudaStream_t);
template void level_apply<float>(hz_handle*, const Level&, const c64*, c64*, int, cudaStream_t);
template void level_residual<double>(hz_handle*, const Level&, const c128*, const c128*, c128*,
                                     int, cudaStream_t);
template void level_residual<float>(hz_handle*, const Level&, const c64*, const c64*, c64*, int,
                                    cudaStream_t);
template void jacobi_steps<double>(hz_handle*, const Level&, const c128*, c128*, c128*, int,
                                   double, int, cudaStream_t);
template void jacobi_steps<float>(hz_handle*, const Level&, const c64*, c64*, c64*, int, double,
                                  int, cudaStream_t);
template void cast_copy<float, double>(const c128*, c64*, size_t, cudaStream_t);
template void cast_copy<double, float>(const c64*, c128*, size_t, cudaStream_t);
template void cast_copy<double, double>(const c128*, c128*, size_t, cudaStream_t);

}  // namespace hz
