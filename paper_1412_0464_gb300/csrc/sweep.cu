// Sweep schedules of Tables 2-3: ForwardSweep, BackwardSweep, MidSolveIn,
// MidSolveOut, SweepingPrecUD and SweepingPrecX.  In the X-sweep the two
// chains that the paper runs simultaneously (forward over 1..j_mid-1 and
// backward over J..j_mid+1, then backward over j_mid-1..1 and forward over
// j_mid+1..J) run on two CUDA streams joined by events; they touch disjoint
// columns of u, disjoint slabs and separate transmission buffers.
#include "hz_internal.h"

namespace hz {

// SubdomSolve (Table 2) on a 2-D slab (twisted block LU along y) or a 3-D
// slab (dense-block LU along z).
template <typename R>
static void sub(hz_handle* h, Level& L, int j, const cplx<R>* f, int a, int b, int at, int bt,
                bool t1, const cplx<R>* B1, bool t2, cplx<R>* B2, bool t3, const cplx<R>* B3,
                bool t4, cplx<R>* B4, cplx<R>* u, int nr, cudaStream_t s) {
  if (L.dim3d)
    subdom_solve3d<R>(h, L, j, f, a, b, at, bt, t1, B1, t2, B2, t3, B3, t4, B4, u, nr, s);
  else
    subdom_solve<R>(h, L, j, f, a, b, at, bt, t1, B1, t2, B2, t3, B3, t4, B4, u, nr, s);
}

template <typename R>
static void forward_sweep(hz_handle* h, Level& L, cplx<R>* u, const cplx<R>* f, int j0, int j1,
                          cplx<R>* B, int nr, cudaStream_t s) {
  const auto& be = L.beta;
  for (int j = j0; j <= j1; ++j)
    sub<R>(h, L, j, f,be[j - 1], be[j], be[j - 1], be[j], j > 1, B, j < L.J, B, false,
                    nullptr, false, nullptr, u, nr, s);
}

template <typename R>
static void backward_sweep(hz_handle* h, Level& L, cplx<R>* u, const cplx<R>* f, int j0, int j1,
                           cplx<R>* B, int nr, cudaStream_t s) {
  const auto& bt = L.beta_t;
  for (int j = j0; j >= j1; --j)
    sub<R>(h, L, j, f,bt[j - 1], bt[j], bt[j - 1], bt[j], false, nullptr, false,
                    nullptr, j < L.J, B, j > 1, B, u, nr, s);
}

template <typename R>
static void mid_solve_in(hz_handle* h, Level& L, cplx<R>* u, const cplx<R>* f, int j, cplx<R>* B1,
                         cplx<R>* B2, int nr, cudaStream_t s) {
  sub<R>(h, L, j, f,L.beta[j - 1], L.beta_t[j], L.beta[j - 1], L.beta_t[j], true, B1,
                  false, nullptr, true, B2, false, nullptr, u, nr, s);
}

template <typename R>
static void mid_solve_out(hz_handle* h, Level& L, cplx<R>* u, const cplx<R>* f, int j, cplx<R>* B1,
                          cplx<R>* B2, int nr, cudaStream_t s) {
  sub<R>(h, L, j, f,L.beta_t[j - 1], L.beta[j], L.beta_t[j - 1], L.beta[j], false,
                  nullptr, true, B1, false, nullptr, true, B2, u, nr, s);
}

// SweepingPrecNX (Table 3): cell boundaries j_cell[0..n_cell] (0, equally
// spaced, J + 1; the listing's j_cell,0 = -1 is read as 0, so that one cell is
// the X-sweep) and cell centres j_mid[1..n_cell].
void nx_layout(int J, int n_cell, std::vector<int>& jc, std::vector<int>& jm) {
  jc.assign(n_cell + 1, 0);
  jm.assign(n_cell + 1, 0);
  for (int m = 1; m < n_cell; ++m) jc[m] = (int)std::lround((double)m * (J + 1) / n_cell);
  jc[n_cell] = J + 1;
  for (int m = 1; m <= n_cell; ++m) {
    jm[m] = (jc[m - 1] + jc[m] + 1) / 2;
    if (!(jc[m - 1] < jm[m] && jm[m] < jc[m]))
      throw Failure(HZ_EINVAL, "NX-sweep: every cell needs at least one subdomain");
  }
}

template <typename R>
__global__ void add_kernel(cplx<R>* u, const cplx<R>* v, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] = u[i] + v[i];
}

// u = P f.  SubdomSolve adds J^T u_d into u; every column receives exactly one
// contribution in each of the two phases of a sweep (the forward phase up to
// g = f - A u, and the phase after it), so each phase stores into its own
// buffer (u, then u2) and u += u2 at the end.
template <typename R>
void sweep_apply(hz_handle* h, Level& L, const cplx<R>* f, cplx<R>* u, int nr, cudaStream_t s) {
  const size_t n = L.size();
  cplx<R>* g = (cplx<R>*)h->pr_g;
  cplx<R>* u2 = (cplx<R>*)h->pr_u2;
  cplx<R>* B1 = (cplx<R>*)h->pr_B1;
  cplx<R>* B2 = (cplx<R>*)h->pr_B2;
  const int J = L.J;
  if (h->p.sweep == HZ_SWEEP_UD) {                  // SweepingPrecUD
    forward_sweep<R>(h, L, u, f, 1, J, B1, nr, s);
    level_residual<R>(h, L, f, u, g, nr, s);
    backward_sweep<R>(h, L, u2, g, J, 1, B1, nr, s);
  } else if (h->p.sweep == HZ_SWEEP_NX) {           // SweepingPrecNX (one stream)
    std::vector<int> jc, jm;
    const int nc = h->p.n_cell;
    nx_layout(J, nc, jc, jm);
    const size_t bs = 2 * (size_t)h->p.max_rhs * L.nt();
    auto Bi = [&](int i) { return (cplx<R>*)h->pr_Bnx + (size_t)i * bs; };
    // first phase: the cell boundaries send their layers into both
    // neighbouring cells, then every cell sweeps towards its centre
    for (int m = 1; m < nc; ++m) mid_solve_out<R>(h, L, u, f, jc[m], Bi(2 * m + 1), Bi(2 * m), nr, s);
    for (int m = 1; m <= nc; ++m) {
      forward_sweep<R>(h, L, u, f, jc[m - 1] + 1, jm[m] - 1, Bi(2 * m - 1), nr, s);
      backward_sweep<R>(h, L, u, f, jc[m] - 1, jm[m] + 1, Bi(2 * m), nr, s);
      mid_solve_in<R>(h, L, u, f, jm[m], Bi(2 * m - 1), Bi(2 * m), nr, s);
    }
    level_residual<R>(h, L, f, u, g, nr, s);
    // second phase: every cell sweeps outwards from its centre, then the cell
    // boundaries take the layers of both neighbouring cells
    for (int m = 1; m <= nc; ++m) {
      mid_solve_out<R>(h, L, u2, g, jm[m], Bi(2 * m), Bi(2 * m - 1), nr, s);
      backward_sweep<R>(h, L, u2, g, jm[m] - 1, jc[m - 1] + 1, Bi(2 * m - 1), nr, s);
      forward_sweep<R>(h, L, u2, g, jm[m] + 1, jc[m] - 1, Bi(2 * m), nr, s);
    }
    for (int m = 1; m < nc; ++m) mid_solve_in<R>(h, L, u2, g, jc[m], Bi(2 * m), Bi(2 * m + 1), nr, s);
  } else {
    const int jm = J / 2 + 1;                        // SweepingPrecX
    cudaStream_t s2 = h->s2;
    HZ_CU(cudaEventRecord(h->evA, s));
    HZ_CU(cudaStreamWaitEvent(s2, h->evA, 0));
    forward_sweep<R>(h, L, u, f, 1, jm - 1, B1, nr, s);
    backward_sweep<R>(h, L, u, f, J, jm + 1, B2, nr, s2);
    HZ_CU(cudaEventRecord(h->evB, s2));
    HZ_CU(cudaStreamWaitEvent(s, h->evB, 0));
    mid_solve_in<R>(h, L, u, f, jm, B1, B2, nr, s);
    level_residual<R>(h, L, f, u, g, nr, s);
    mid_solve_out<R>(h, L, u2, g, jm, B2, B1, nr, s);
    HZ_CU(cudaEventRecord(h->evA, s));
    HZ_CU(cudaStreamWaitEvent(s2, h->evA, 0));
    backward_sweep<R>(h, L, u2, g, jm - 1, 1, B1, nr, s);
    forward_sweep<R>(h, L, u2, g, jm + 1, J, B2, nr, s2);
    HZ_CU(cudaEventRecord(h->evB, s2));
    HZ_CU(cudaStreamWaitEvent(s, h->evB, 0));
  }
  add_kernel<R><<<cdiv(n * nr, 256), 256, 0, s>>>(u, u2, n * nr);
  h->launches++;
  HZ_CU(cudaGetLastError());
}

// Two-grid sweeping preconditioner (Section 4): u = 0; nu omega-Jacobi steps;
// r_c = R (f - A u); e_c = P_X r_c (or P_UD) on the coarse operator; u += P e_c;
// nu omega-Jacobi steps.
template <typename R>
static void tgsp(hz_handle* h, const cplx<R>* f, cplx<R>* u, int nr, cudaStream_t s) {
  Level& F = h->fine;
  Level& C = h->coarse;
  const size_t nf = F.size();
  cplx<R>* t = (cplx<R>*)h->tg_t;
  HZ_CU(cudaMemsetAsync(u, 0, sizeof(cplx<R>) * nf * nr, s));
  jacobi_steps<R>(h, F, f, u, t, h->p.nu, h->p.omega_jac, nr, s);
  level_residual<R>(h, F, f, u, t, nr, s);
  restrict_residual<R>(h, F, C, t, (cplx<R>*)h->pr_r, nr, s);
  sweep_apply<R>(h, C, (const cplx<R>*)h->pr_r, (cplx<R>*)h->pr_u, nr, s);
  prolong_add<R>(h, F, C, (const cplx<R>*)h->pr_u, u, nr, s);
  jacobi_steps<R>(h, F, f, u, t, h->p.nu, h->p.omega_jac, nr, s);
}

template <typename R>
static void precond_t(hz_handle* h, const c128* r, c128* z, int nr, cudaStream_t s) {
  Level& F = h->fine;
  const size_t n = F.size();
  if (!h->p.two_grid) {
    if (sizeof(R) == 8) {
      sweep_apply<R>(h, F, (const cplx<R>*)r, (cplx<R>*)z, nr, s);
    } else {
      cast_copy<R, double>(r, (cplx<R>*)h->pr_r, n * nr, s);
      sweep_apply<R>(h, F, (const cplx<R>*)h->pr_r, (cplx<R>*)h->pr_u, nr, s);
      cast_copy<double, R>((const cplx<R>*)h->pr_u, z, n * nr, s);
    }
    return;
  }
  if (sizeof(R) == 8) {
    tgsp<R>(h, (const cplx<R>*)r, (cplx<R>*)z, nr, s);
  } else {
    cast_copy<R, double>(r, (cplx<R>*)h->tg_r, n * nr, s);
    tgsp<R>(h, (const cplx<R>*)h->tg_r, (cplx<R>*)h->tg_u, nr, s);
    cast_copy<double, R>((const cplx<R>*)h->tg_u, z, n * nr, s);
  }
}

void precond_apply(hz_handle* h, const c128* r, c128* z, int nr, cudaStream_t s) {
  if (h->p.precision == HZ_MIXED)
    precond_t<float>(h, r, z, nr, s);
  else
    precond_t<double>(h, r, z, nr, s);
}

template void sweep_apply<float>(hz_handle*, Level&, const c64*, c64*, int, cudaStream_t);
template void sweep_apply<double>(hz_handle*, Level&, const c128*, c128*, int, cudaStream_t);

}  // namespace hz
