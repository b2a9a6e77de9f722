// Matrix-free 3-D Helmholtz operator kernels.
//
// Fine level: the 7-point analogue of Eq. 40 multiplied by h^3, each second
// difference divided by the PML factors of the other two axes:
//   (A u)_i = h [ (1/(a2 a3)) (-a1_{x-1/2} u_{x-1} + (a1_{x-1/2} + a1_{x+1/2}) u - a1_{x+1/2} u_{x+1})
//               + (1/(a1 a3)) (same along y) + (1/(a1 a2)) (same along z) ]
//             - h^3 omega^2 m_i / (a1 a2 a3) u_i,
// Dirichlet zeros outside.  Where alpha = 1 exactly at the node and at the
// adjacent cells of all three axes the row is real:
//   (A u)_i = h [ (6 - h^2 omega^2 m_i) u_i - (sum of the six neighbours) ].
// Coarse level: the stored 27-point FE stencil (Appendix A, Eq. 63), planes
// q = (dz+1) 9 + (dy+1) 3 + (dx+1), layout [27][nz][ny][nx].
// Modes as in the 2-D kernels: 0 y = A u, 1 y = f - A u,
// 2 (omega-Jacobi) y = u + omega_J (f - A u) / diag(A).
#include "hz_internal.h"

namespace hz {

namespace {

template <typename R> struct Tab3;
template <> struct Tab3<double> {
  static const double* beta(const AxisTables& a) { return a.beta; }
  static const c128* inode(const AxisTables& a) { return a.ia_node; }
  static const c128* cell(const AxisTables& a) { return a.a_cell; }
  static const double* m(const Level& L) { return L.m; }
  static const c128* st(const Level& L) { return L.st128; }
};
template <> struct Tab3<float> {
  static const float* beta(const AxisTables& a) { return a.beta32; }
  static const c64* inode(const AxisTables& a) { return a.ia_node32; }
  static const c64* cell(const AxisTables& a) { return a.a_cell32; }
  static const float* m(const Level& L) { return L.m32; }
  static const c64* st(const Level& L) { return L.st64; }
};

template <typename R>
struct Op3Args {
  int mode, nx, ny, nz;
  R hh, h2w2, omega_jac;               // h (the h^(d-2) factor), h^2 omega^2
  const R* m;
  const cplx<R>* ia[3];                // 1/alpha at unknowns, x y z
  const cplx<R>* ac[3];                // alpha at cell midpoints, x y z
  const R* beta[3];                    // sponge profiles, x y z (null: PML)
  const cplx<R>* st;                   // stored 27-point planes or null
  int lo[3], hi[3];                    // real-coefficient interior box
  const cplx<R>* f;
  const cplx<R>* u;
  cplx<R>* y;
};

template <typename R, bool STORED>
__global__ void __launch_bounds__(128) op3d_kernel(Op3Args<R> a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int yy = blockIdx.y;
  const int z = blockIdx.z % a.nz, r = blockIdx.z / a.nz;
  if (x >= a.nx) return;
  const size_t n = (size_t)a.nx * a.ny * a.nz;
  const size_t sxy = (size_t)a.nx * a.ny;
  const cplx<R>* U = a.u + (size_t)r * n;
  const size_t c = ((size_t)z * a.ny + yy) * a.nx + x;
  const size_t i = (size_t)r * n + c;
  const cplx<R> zero = mk<R>(0, 0);
  const cplx<R> uc = U[c];
  cplx<R> au, dg;
  if (STORED) {
    au = zero;
    const size_t plane = n;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = z + dz;
      if (zz < 0 || zz >= a.nz) continue;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int y2 = yy + dy;
        if (y2 < 0 || y2 >= a.ny) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int x2 = x + dx;
          if (x2 < 0 || x2 >= a.nx) continue;
          const int q = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
          cfma(au, a.st[(size_t)q * plane + c], U[((size_t)zz * a.ny + y2) * a.nx + x2]);
        }
      }
    }
    dg = a.st[(size_t)13 * plane + c];
  } else {
    const cplx<R> ul = x > 0 ? U[c - 1] : zero, ur = x < a.nx - 1 ? U[c + 1] : zero;
    const cplx<R> ud = yy > 0 ? U[c - a.nx] : zero, uu = yy < a.ny - 1 ? U[c + a.nx] : zero;
    const cplx<R> ub = z > 0 ? U[c - sxy] : zero, ut = z < a.nz - 1 ? U[c + sxy] : zero;
    const R mm = a.h2w2 * a.m[c];
    if (x >= a.lo[0] && x <= a.hi[0] && yy >= a.lo[1] && yy <= a.hi[1] && z >= a.lo[2] &&
        z <= a.hi[2]) {
      const R cc = (R)6 - mm;
      au = mk<R>(a.hh * (cc * uc.re - (((ul.re + ur.re) + (ud.re + uu.re)) + (ub.re + ut.re))),
                 a.hh * (cc * uc.im - (((ul.im + ur.im) + (ud.im + uu.im)) + (ub.im + ut.im))));
      dg = mk<R>(a.hh * cc, (R)0);
    } else {
      const cplx<R> i1 = a.ia[0][x], i2 = a.ia[1][yy], i3 = a.ia[2][z];
      const cplx<R> xl = a.ac[0][x], xr = a.ac[0][x + 1];
      const cplx<R> yl = a.ac[1][yy], yr = a.ac[1][yy + 1];
      const cplx<R> zl = a.ac[2][z], zr = a.ac[2][z + 1];
      const cplx<R> tx = (xl + xr) * uc - xl * ul - xr * ur;
      const cplx<R> ty = (yl + yr) * uc - yl * ud - yr * uu;
      const cplx<R> tz = (zl + zr) * uc - zl * ub - zr * ut;
      const cplx<R> s23 = i2 * i3, s13 = i1 * i3, s12 = i1 * i2;
      cplx<R> mass = mm * (s12 * i3);
      if (a.beta[0])                      // sponge: k^2 (1 + i beta)^2
        mass = mass * sponge_s<R>(a.beta[0][x] + a.beta[1][yy] + a.beta[2][z]);
      au = a.hh * (s23 * tx + s13 * ty + s12 * tz - mass * uc);
      dg = a.hh * (s23 * (xl + xr) + s13 * (yl + yr) + s12 * (zl + zr) - mass);
    }
  }
  if (a.mode == 0) {
    a.y[i] = au;
  } else if (a.mode == 1) {
    a.y[i] = a.f[i] - au;
  } else {
    a.y[i] = uc + a.omega_jac * ((a.f[i] - au) * cinv(dg));
  }
}

}  // namespace

template <typename R>
void launch_op3d(hz_handle* h, const Level& L, int mode, const cplx<R>* f, const cplx<R>* u,
                 cplx<R>* y, int n_rhs, double omega_jac, cudaStream_t s) {
  Op3Args<R> a{};
  a.mode = mode;
  a.nx = L.nx; a.ny = L.ny; a.nz = L.nz;
  a.hh = (R)L.h;
  a.h2w2 = (R)(L.h * L.h * h->p.omega * h->p.omega);
  a.omega_jac = (R)omega_jac;
  a.f = f; a.u = u; a.y = y;
  const AxisTables* ax[3] = {&L.ax, &L.ay, &L.az};
  for (int l = 0; l < 3; ++l) {
    a.lo[l] = ax[l]->in_lo;
    a.hi[l] = ax[l]->in_hi;
    if (!L.fe) {
      a.ia[l] = Tab3<R>::inode(*ax[l]);
      a.ac[l] = Tab3<R>::cell(*ax[l]);
      a.beta[l] = Tab3<R>::beta(*ax[l]);
    }
  }
  if (!L.fe) a.m = Tab3<R>::m(L);
  const dim3 grid(cdiv(L.nx, 128), L.ny, L.nz * n_rhs);
  const double el = sizeof(cplx<R>), dofs = (double)L.size() * n_rhs;
  const double coef = L.fe ? 27.0 * el : (double)sizeof(R);
  const double bytes = dofs * (2.0 * el + (mode >= 1 ? el : 0.0) + coef);
  const char* tag = sizeof(R) == 4 ? "stencil_c64" : "stencil_c128";
  if (L.fe) {
    a.st = Tab3<R>::st(L);
    timed(h, tag, bytes, s, [&] { op3d_kernel<R, true><<<grid, 128, 0, s>>>(a); });
  } else {
    timed(h, tag, bytes, s, [&] { op3d_kernel<R, false><<<grid, 128, 0, s>>>(a); });
  }
  h->launches++;
  HZ_CU(cudaGetLastError());
}

template void launch_op3d<float>(hz_handle*, const Level&, int, const c64*, const c64*, c64*, int,
                                 double, cudaStream_t);
template void launch_op3d<double>(hz_handle*, const Level&, int, const c128*, const c128*, c128*,
                                  int, double, cudaStream_t);

}  // namespace hz
