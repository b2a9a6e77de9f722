// Adjoint gradient of the receiver misfit
//   Phi(m) = 1/2 sum_s sum_q |u_s(x_q) - d_{s,q}|^2,   A(m) u_s = e_{src_s}.
// Only the mass term of Eq. 40 depends on m (k^2 = omega^2 m s, s = (1 + i beta)^2
// in a sponge layer of Section 2.1, else 1), so dA/dm_i = -omega^2 w_i e_i e_i^T
// with w_i = h^d s_i / (alpha_x alpha_y)_i, the PML and sponge held fixed.  A is complex symmetric (Eq. 40), so the adjoint field solves
// A mu_s = conj(R^T r_s) with the same preconditioner and factors, and
//   dPhi/dm_i = omega^2 Re(w_i sum_s mu_{s,i} u_{s,i}).
// Sources are taken in batches of max_rhs: one forward and one adjoint
// multi-right-hand-side GMRES solve per batch.
#include "hz_internal.h"

#include <algorithm>
#include <vector>

namespace hz {

namespace {

__global__ void point_sources_kernel(c128* b, size_t n, const int* src, int nb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nb) b[(size_t)k * n + src[k]] = mk<double>(1.0, 0.0);
}

// One thread per right-hand side, receivers in order (deterministic; repeated
// receivers add up): b_k[rec_q] += conj(u_k[rec_q] - d_kq), phi_k = sum |r|^2 / 2.
__global__ void receiver_residual_kernel(const c128* u, size_t n, const int* rec, int n_rec,
                                         const c128* d, c128* b, double* phi, int nb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  const c128* uk = u + (size_t)k * n;
  c128* bk = b + (size_t)k * n;
  const c128* dk = d + (size_t)k * n_rec;
  double acc = 0.0;
  for (int q = 0; q < n_rec; ++q) {
    const int i = rec[q];
    const double rr = uk[i].re - dk[q].re, ri = uk[i].im - dk[q].im;
    acc += rr * rr + ri * ri;
    bk[i].re += rr;
    bk[i].im -= ri;
  }
  phi[k] = 0.5 * acc;
}

// grad_i += omega^2 Re( h^d s_i / (alpha_x alpha_y [alpha_z])_i * sum_k mu_k,i u_k,i )
// (scale = omega^2 h^d; az and bz are null in 2-D, bx null without a sponge)
__global__ void grad_accumulate_kernel(const c128* u, const c128* mu, int nb, int nx, int ny,
                                       int nz, const c128* ax, const c128* ay, const c128* az,
                                       const double* bx, const double* by, const double* bz,
                                       double scale, double* grad) {
  const size_t n = (size_t)nx * ny * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    c128 acc = mk<double>(0.0, 0.0);
    for (int k = 0; k < nb; ++k) cfma(acc, mu[(size_t)k * n + i], u[(size_t)k * n + i]);
    const size_t iyz = i / nx;
    const int ix = (int)(i - iyz * nx);
    const int iy = (int)(iyz % ny), iz = (int)(iyz / ny);
    c128 pa = ax[ix] * ay[iy];
    if (az) pa = pa * az[iz];
    c128 w = cinv(pa);
    if (bx) w = w * sponge_s(bx[ix] + by[iy] + (bz ? bz[iz] : 0.0));
    grad[i] += scale * (w * acc).re;
  }
}

}  // namespace

void misfit_grad(hz_handle* h, const int* src, int n_src, const int* rec, int n_rec,
                 const c128* d, double* grad, double* phi_out, cudaStream_t s) {
  Level& F = h->fine;
  const size_t n = F.size();
  // Indices are validated on the host before any kernel uses them.
  std::vector<int> hs(n_src), hr(n_rec);
  HZ_CU(cudaMemcpyAsync(hs.data(), src, sizeof(int) * n_src, cudaMemcpyDeviceToHost, s));
  if (n_rec > 0)
    HZ_CU(cudaMemcpyAsync(hr.data(), rec, sizeof(int) * n_rec, cudaMemcpyDeviceToHost, s));
  HZ_CU(cudaStreamSynchronize(s));
  for (int v : hs)
    if (v < 0 || (size_t)v >= n) throw Failure(HZ_EINVAL, "source index outside the grid");
  for (int v : hr)
    if (v < 0 || (size_t)v >= n) throw Failure(HZ_EINVAL, "receiver index outside the grid");

  const int R = h->p.max_rhs;
  if (!h->gr_b) {   // allocated once, on the first gradient call
    h->gr_b = (c128*)dmalloc(sizeof(c128) * n * R);
    h->gr_u = (c128*)dmalloc(sizeof(c128) * n * R);
    h->gr_mu = (c128*)dmalloc(sizeof(c128) * n * R);
    h->gr_phi = (double*)dmalloc(sizeof(double) * R);
  }
  HZ_CU(cudaMemsetAsync(grad, 0, sizeof(double) * n, s));
  const double scale =
      h->p.omega * h->p.omega * F.h * F.h * (F.dim3d ? F.h : 1.0);   // omega^2 h^d
  double phi = 0.0;
  int iters_max = 0;
  double relres_max = 0.0;
  long long applies = 0;
  bool conv = true;
  auto solve = [&](const c128* b, c128* u, int nb) {
    h->stats.precond_applies = 0;
    try {
      gmres_solve(h, b, u, nb, s);
    } catch (const Failure& f) {
      if (f.st != HZ_ENOTCONV) throw;
      conv = false;
    }
    iters_max = std::max(iters_max, h->stats.iters_max);
    relres_max = std::max(relres_max, h->stats.relres_max);
    applies += h->stats.precond_applies;
  };
  std::vector<double> hphi(R);
  for (int s0 = 0; s0 < n_src; s0 += R) {
    const int nb = std::min(R, n_src - s0);
    HZ_CU(cudaMemsetAsync(h->gr_b, 0, sizeof(c128) * n * nb, s));
    point_sources_kernel<<<1, 64, 0, s>>>(h->gr_b, n, src + s0, nb);
    h->launches++;
    solve(h->gr_b, h->gr_u, nb);
    HZ_CU(cudaMemsetAsync(h->gr_b, 0, sizeof(c128) * n * nb, s));
    receiver_residual_kernel<<<1, 64, 0, s>>>(h->gr_u, n, rec, n_rec, d + (size_t)s0 * n_rec,
                                              h->gr_b, h->gr_phi, nb);
    h->launches++;
    solve(h->gr_b, h->gr_mu, nb);
    grad_accumulate_kernel<<<4 * h->sms, 256, 0, s>>>(
        h->gr_u, h->gr_mu, nb, F.nx, F.ny, F.nz, F.ax.a_node, F.ay.a_node,
        F.dim3d ? F.az.a_node : nullptr, F.ax.beta, F.ay.beta, F.dim3d ? F.az.beta : nullptr,
        scale, grad);
    h->launches++;
    HZ_CU(cudaMemcpyAsync(hphi.data(), h->gr_phi, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    HZ_CU(cudaStreamSynchronize(s));
    HZ_CU(cudaGetLastError());
    for (int k = 0; k < nb; ++k) phi += hphi[k];
  }
  h->stats.n_rhs = n_src;
  h->stats.iters_max = iters_max;
  h->stats.relres_max = relres_max;
  h->stats.precond_applies = applies;
  *phi_out = phi;
  if (!conv) throw Failure(HZ_ENOTCONV, "GMRES did not reach the tolerance within max_iter");
}

}  // namespace hz
