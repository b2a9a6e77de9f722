// Restarted right-preconditioned GMRES(m) in FP64 (the outer Krylov method in
// which the paper applies its preconditioners, Section 4; stopping rule
// ||b - A u|| / ||b|| <= tol, Section 6.1).  Arnoldi with classical
// Gram-Schmidt and one re-orthogonalisation (CGS2); the preconditioned
// vectors Z_j = M V_j are kept so that the update is x += Z y.  The
// Hessenberg column, Givens rotations and the triangular solve run in a
// one-block kernel per right-hand side; the host reads only the residual
// estimates (8 bytes per right-hand side) to decide when to stop.
#include "hz_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace hz {

constexpr int kRedBlocks = 296;   // 2 x 148 blocks per right-hand side
constexpr int kRedThreads = 256;
constexpr int kMaxRhsThreads = 64;   // one thread per right-hand side (max_rhs <= 64)

// partial[r][i][blk] = sum over the block's chunk of conj(V_i) . w   (i < nv)
__global__ void __launch_bounds__(kRedThreads) multi_dot_kernel(const c128* __restrict__ V,
                                                                size_t vstride, int nv,
                                                                const c128* __restrict__ w,
                                                                size_t n, int nr,
                                                                double* __restrict__ partial) {
  const int r = blockIdx.y;
  __shared__ double sh[2][kRedThreads];
  const c128* wr = w + (size_t)r * n;
  for (int i = 0; i < nv; ++i) {
    const c128* v = V + (size_t)i * vstride + (size_t)r * n;
    double re = 0, im = 0;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
      c128 a = v[x], b = wr[x];
      re = fma(a.re, b.re, re); re = fma(a.im, b.im, re);
      im = fma(a.re, b.im, im); im = fma(-a.im, b.re, im);
    }
    sh[0][threadIdx.x] = re;
    sh[1][threadIdx.x] = im;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
        sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      size_t o = (((size_t)r * nv + i) * gridDim.x + blockIdx.x) * 2;
      partial[o] = sh[0][0];
      partial[o + 1] = sh[1][0];
    }
    __syncthreads();
  }
}

// out[r][i] (+)= sum_blk partial[r][i][blk]  (fixed order: deterministic)
// One warp per (rhs, vector): lane l sums partials l, l + 32, ..., then a
// shuffle tree (fixed order, so the result is repeatable).
__global__ void reduce_partials_kernel(const double* partial, int nblk, int nv, int nr, c128* out,
                                       int ostride) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= nv * nr) return;
  const double2* p = reinterpret_cast<const double2*>(partial + (size_t)t * nblk * 2);
  double re = 0, im = 0;
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = p[b];
    re += v.x;
    im += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    const int r = t / nv, i = t - r * nv;
    out[(size_t)r * ostride + i] = mk(re, im);
  }
}

// hc[r][i] += hc2[r][i] for i < nv
__global__ void add_coeffs_kernel(c128* hc, const c128* hc2, int hstride, int nv, int nr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nr) return;
  int r = t / nv, i = t - r * nv;
  hc[(size_t)r * hstride + i] = hc[(size_t)r * hstride + i] + hc2[(size_t)r * hstride + i];
}

// w -= sum_i h[r][i] V_i
__global__ void multi_axpy_kernel(const c128* __restrict__ V, size_t vstride, int nv,
                                  const c128* __restrict__ hc, int hstride, c128* __restrict__ w,
                                  size_t n) {
  const int r = blockIdx.y;
  size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= n) return;
  c128 acc = w[(size_t)r * n + x];
  for (int i = 0; i < nv; ++i) {
    c128 c = hc[(size_t)r * hstride + i];
    c128 v = V[(size_t)i * vstride + (size_t)r * n + x];
    acc.re -= c.re * v.re - c.im * v.im;
    acc.im -= c.re * v.im + c.im * v.re;
  }
  w[(size_t)r * n + x] = acc;
}

// x += sum_i y[r][i] Z_i
__global__ void basis_update_kernel(const c128* __restrict__ Z, size_t zstride, int nv,
                                    const c128* __restrict__ y, int ystride, c128* __restrict__ x,
                                    size_t n) {
  const int r = blockIdx.y;
  size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i0 >= n) return;
  c128 acc = x[(size_t)r * n + i0];
  for (int i = 0; i < nv; ++i) cfma(acc, y[(size_t)r * ystride + i], Z[(size_t)i * zstride + (size_t)r * n + i0]);
  x[(size_t)r * n + i0] = acc;
}

// V_{j+1} = w / ||w|| (norm from hcol[r][j+1], real part)
__global__ void scale_kernel(const c128* __restrict__ w, c128* __restrict__ v, size_t n,
                             const c128* __restrict__ hc, int hstride, int idx) {
  const int r = blockIdx.y;
  size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= n) return;
  double nrm = hc[(size_t)r * hstride + idx].re;
  double s = nrm > 0 ? 1.0 / nrm : 0.0;
  c128 a = w[(size_t)r * n + x];
  v[(size_t)r * n + x] = mk(a.re * s, a.im * s);
}

__global__ void norm_from_dot_kernel(c128* hc, int hstride, int idx, int nr) {
  int r = threadIdx.x;
  if (r < nr) {
    // a NaN sum stays NaN (a NaN norm must not read as zero, i.e. converged)
    double v = hc[(size_t)r * hstride + idx].re;
    hc[(size_t)r * hstride + idx] = mk(isnan(v) ? v : sqrt(v > 0 ? v : 0.0), 0.0);
  }
}

struct ArnoldiState {
  c128* H;      // [nr][(m+1)*m] column-major
  double* cs;   // [nr][m]
  c128* sn;     // [nr][m]
  c128* g;      // [nr][m+1]
  double* res;  // [nr] |g_{j+1}|
  int* kdone;   // [nr] columns used by the current cycle (frozen once converged)
};

// Apply the previous rotations to column j (in hc[r][0..j+1]), form a new
// rotation that annihilates H[j+1][j], update g.  One thread per right-hand side.
__global__ void arnoldi_update_kernel(ArnoldiState a, const c128* hc, int hstride, int m, int j,
                                      int nr, const double* bnorm, double tol) {
  int r = threadIdx.x;
  if (r >= nr) return;
  if (a.kdone[r] < j) return;   // converged earlier in this cycle: frozen
  c128* H = a.H + (size_t)r * (m + 1) * m;
  c128* col = H + (size_t)j * (m + 1);
  for (int i = 0; i <= j + 1; ++i) col[i] = hc[(size_t)r * hstride + i];
  double* cs = a.cs + (size_t)r * m;
  c128* sn = a.sn + (size_t)r * m;
  c128* g = a.g + (size_t)r * (m + 1);
  for (int i = 0; i < j; ++i) {
    c128 t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = (-cconj(sn[i])) * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  c128 x = col[j], y = col[j + 1];
  double ax = sqrt(cabs2(x)), ay = sqrt(cabs2(y));
  double c;
  c128 s, rr;
  if (ay == 0) { c = 1; s = mk(0.0, 0.0); rr = x; }
  else if (ax == 0) { c = 0; s = mk(1.0, 0.0); rr = y; }
  else {
    double nu = hypot(ax, ay);
    c128 ph = mk(x.re / ax, x.im / ax);
    c = ax / nu;
    s = (1.0 / nu) * (ph * cconj(y));
    rr = nu * ph;
  }
  cs[j] = c; sn[j] = s;
  col[j] = rr; col[j + 1] = mk(0.0, 0.0);
  c128 gj = g[j];
  g[j + 1] = (-cconj(s)) * gj;
  g[j] = c * gj;
  a.res[r] = sqrt(cabs2(g[j + 1]));
  a.kdone[r] = j + 1;
  if (a.res[r] <= tol * bnorm[r]) a.kdone[r] = -(j + 1);   // converged: freeze (negative)
}

// Back substitution H y = g over the k columns of the cycle.
__global__ void solve_upper_kernel(ArnoldiState a, int m, int nr, c128* y) {
  int r = threadIdx.x;
  if (r >= nr) return;
  int k = a.kdone[r];
  if (k < 0) k = -k;
  const c128* H = a.H + (size_t)r * (m + 1) * m;
  const c128* g = a.g + (size_t)r * (m + 1);
  c128* yr = y + (size_t)r * m;
  for (int i = 0; i < m; ++i) yr[i] = mk(0.0, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    c128 acc = g[i];
    for (int c = i + 1; c < k; ++c) {
      c128 hv = H[(size_t)c * (m + 1) + i];
      acc.re -= hv.re * yr[c].re - hv.im * yr[c].im;
      acc.im -= hv.re * yr[c].im + hv.im * yr[c].re;
    }
    yr[i] = acc * cinv(H[(size_t)i * (m + 1) + i]);
  }
}

__global__ void cycle_init_kernel(ArnoldiState a, int m, int nr, const c128* hc, int hstride,
                                  int idx) {
  int r = threadIdx.x;
  if (r >= nr) return;
  c128* g = a.g + (size_t)r * (m + 1);
  for (int i = 0; i <= m; ++i) g[i] = mk(0.0, 0.0);
  g[0] = hc[(size_t)r * hstride + idx];   // beta = ||r0||
  a.kdone[r] = 0;
}

struct Gm {
  hz_handle* h;
  size_t n;
  int nr, m;
  cudaStream_t s;
  // out[r*ostride + i] = <V_i, w_r>, i < nv
  void dots(const c128* V, size_t vstride, int nv, const c128* w, c128* out, int ostride) {
    dim3 grid(kRedBlocks, nr);
    multi_dot_kernel<<<grid, kRedThreads, 0, s>>>(V, vstride, nv, w, n, nr, h->red);
    reduce_partials_kernel<<<cdiv(nv * nr, 4), 128, 0, s>>>(h->red, kRedBlocks, nv, nr, out, ostride);
    h->launches += 2;
  }
};

// Scratch needed by the reductions: kRedBlocks * 2 doubles per (rhs, vector).
size_t gmres_red_doubles(int m, int nr) { return (size_t)kRedBlocks * 2 * (m + 2) * nr; }

void gmres_solve(hz_handle* h, const c128* f, c128* u, int nr, cudaStream_t s) {
  Level& F = h->fine;
  const size_t n = F.size();
  const int m = h->p.gmres_m;
  const size_t vs = n * nr;   // stride between basis vectors
  Gm gm{h, n, nr, m, s};
  // Arnoldi state for max_rhs right-hand sides: allocated by the first solve
  // and kept by the handle (a solve allocates nothing after that)
  const int R = h->p.max_rhs;
  const size_t b_H = sizeof(c128) * R * (m + 1) * m, b_cs = sizeof(double) * R * m;
  const size_t b_sn = sizeof(c128) * R * m, b_g = sizeof(c128) * R * (m + 1);
  const size_t b_res = sizeof(double) * R, b_kd = sizeof(int) * R * 2;
  const size_t b_y = sizeof(c128) * R * m, b_bn = sizeof(double) * R;
  if (!h->gm_state) h->gm_state = dmalloc(b_H + b_cs + b_sn + b_g + b_res + b_kd + b_y + b_bn);
  unsigned char* gp = (unsigned char*)h->gm_state;
  ArnoldiState st;
  st.H = (c128*)gp;                          gp += b_H;
  st.g = (c128*)gp;                          gp += b_g;
  st.sn = (c128*)gp;                         gp += b_sn;
  c128* y = (c128*)gp;                       gp += b_y;
  st.cs = (double*)gp;                       gp += b_cs;
  st.res = (double*)gp;                      gp += b_res;
  double* bnorm_d = (double*)gp;             gp += b_bn;
  st.kdone = (int*)gp;
  const int hs = m + 2;
  c128* hc = h->hcol;                    // [nr][hs]
  c128* hc2 = h->hcol + (size_t)nr * hs; // [nr][hs]
  const dim3 eg(cdiv(n, 256), nr);
  const double tol = h->p.tol;

  auto norms = [&](const c128* v, std::vector<double>& out) {
    gm.dots(v, vs, 1, v, hc, hs);
    norm_from_dot_kernel<<<1, kMaxRhsThreads, 0, s>>>(hc, hs, 0, nr);
    std::vector<c128> hb((size_t)nr * hs);
    HZ_CU(cudaMemcpyAsync(hb.data(), hc, sizeof(c128) * nr * hs, cudaMemcpyDeviceToHost, s));
    HZ_CU(cudaStreamSynchronize(s));
    out.resize(nr);
    for (int r = 0; r < nr; ++r) out[r] = hb[(size_t)r * hs].re;
  };

  std::vector<double> bnorm, rnorm;
  norms(f, bnorm);
  HZ_CU(cudaMemcpyAsync(bnorm_d, bnorm.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s));
  HZ_CU(cudaMemsetAsync(u, 0, sizeof(c128) * n * nr, s));
  HZ_CU(cudaMemcpyAsync(h->R, f, sizeof(c128) * n * nr, cudaMemcpyDeviceToDevice, s));
  std::vector<int> iters(nr, 0);
  std::vector<double> relres(nr, 1.0);
  std::vector<char> active(nr, 1);
  for (int r = 0; r < nr; ++r)
    if (bnorm[r] == 0) { relres[r] = 0; active[r] = 0; }
  std::vector<double> res(nr);
  std::vector<int> kd(nr);
  int cycles = 0;
  while (true) {
    bool any = false;
    int maxit = 0;
    for (int r = 0; r < nr; ++r) { any = any || active[r]; maxit = std::max(maxit, iters[r]); }
    if (!any || maxit >= h->p.max_iter) break;
    // beta = ||R||, V_0 = R / beta; inactive right-hand sides start with g = 0
    gm.dots(h->R, vs, 1, h->R, hc, hs);
    norm_from_dot_kernel<<<1, kMaxRhsThreads, 0, s>>>(hc, hs, 0, nr);
    scale_kernel<<<eg, 256, 0, s>>>(h->R, h->V, n, hc, hs, 0);
    cycle_init_kernel<<<1, kMaxRhsThreads, 0, s>>>(st, m, nr, hc, hs, 0);
    h->launches += 3;
    for (int r = 0; r < nr; ++r)
      if (!active[r]) HZ_CU(cudaMemsetAsync(st.g + (size_t)r * (m + 1), 0, sizeof(c128), s));
    int kmax = 0;
    for (int j = 0; j < m; ++j) {
      c128* Vj = h->V + (size_t)j * vs;
      c128* Zj = h->Z + (size_t)j * vs;
      precond_graphed(h, Vj, Zj, nr, s);
      h->stats.precond_applies++;
      apply_fine64(h, Zj, h->W, nr, s);
      gm.dots(h->V, vs, j + 1, h->W, hc, hs);                       // h1 = V^H w
      multi_axpy_kernel<<<eg, 256, 0, s>>>(h->V, vs, j + 1, hc, hs, h->W, n);
      gm.dots(h->V, vs, j + 1, h->W, hc2, hs);                      // h2 = V^H w
      multi_axpy_kernel<<<eg, 256, 0, s>>>(h->V, vs, j + 1, hc2, hs, h->W, n);
      add_coeffs_kernel<<<cdiv((j + 1) * nr, 64), 64, 0, s>>>(hc, hc2, hs, j + 1, nr);
      gm.dots(h->W, vs, 1, h->W, hc + (j + 1), hs);                 // ||w||^2
      norm_from_dot_kernel<<<1, kMaxRhsThreads, 0, s>>>(hc, hs, j + 1, nr);
      scale_kernel<<<eg, 256, 0, s>>>(h->W, h->V + (size_t)(j + 1) * vs, n, hc, hs, j + 1);
      arnoldi_update_kernel<<<1, kMaxRhsThreads, 0, s>>>(st, hc, hs, m, j, nr, bnorm_d, tol);
      h->launches += 7;
      HZ_CU(cudaMemcpyAsync(kd.data(), st.kdone, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
      HZ_CU(cudaStreamSynchronize(s));
      HZ_CU(cudaGetLastError());
      kmax = j + 1;
      bool all_frozen = true;
      int maxit2 = 0;
      for (int r = 0; r < nr; ++r) {
        if (kd[r] >= 0) all_frozen = false;
        int used = iters[r] + (active[r] ? (kd[r] < 0 ? -kd[r] : kd[r]) : 0);
        maxit2 = std::max(maxit2, used);
      }
      if (all_frozen || maxit2 >= h->p.max_iter) break;
    }
    solve_upper_kernel<<<1, kMaxRhsThreads, 0, s>>>(st, m, nr, y);
    basis_update_kernel<<<eg, 256, 0, s>>>(h->Z, vs, kmax, y, m, u, n);
    level_residual<double>(h, F, f, u, h->R, nr, s);
    h->launches += 2;
    HZ_CU(cudaMemcpyAsync(kd.data(), st.kdone, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    norms(h->R, rnorm);
    for (int r = 0; r < nr; ++r) {
      if (!active[r]) continue;
      iters[r] += kd[r] < 0 ? -kd[r] : kd[r];
      relres[r] = bnorm[r] > 0 ? rnorm[r] / bnorm[r] : 0.0;
      if (!std::isfinite(relres[r]))
        throw Failure(HZ_EINACCURATE, "non-finite residual in GMRES (right-hand side " +
                                          std::to_string(r) + ")");
      if (relres[r] <= tol) active[r] = 0;
    }
    ++cycles;
  }
  check_dev_flag(h, s);
  h->stats.n_rhs = nr;
  h->stats.iters_max = 0;
  h->stats.relres_max = 0;
  bool conv = true;
  for (int r = 0; r < nr; ++r) {
    h->stats.iters_max = std::max(h->stats.iters_max, iters[r]);
    h->stats.relres_max = std::max(h->stats.relres_max, relres[r]);
    conv = conv && relres[r] <= tol;
  }
  if (!conv) throw Failure(HZ_ENOTCONV, "GMRES did not reach the tolerance within max_iter");
}

// The preconditioner application is a fixed sequence of a few hundred
// launches (sweeps over J slabs, each a chain of substitution kernels, plus
// the two-grid transfers), identical for every GMRES iteration with the same
// buffers.  It is captured once per (input, output, n_rhs) as a CUDA graph
// and replayed, which removes the per-launch host cost; the X-sweep's second
// stream joins the capture through its fork / join events.  The first
// application for an n_rhs runs uncaptured (it makes the lazy allocations),
// and timing (per-kernel events) or HZ_TEST_NO_GRAPH=1 bypass the graphs.
void precond_graphed(hz_handle* h, const c128* in, c128* out, int nr, cudaStream_t s) {
  const bool warm = std::find(h->pwarm.begin(), h->pwarm.end(), nr) != h->pwarm.end();
  if (h->timing.on || !warm || test_hook("HZ_TEST_NO_GRAPH") > 0) {
    precond_apply(h, in, out, nr, s);
    if (!warm) h->pwarm.push_back(nr);
    return;
  }
  hz_handle::PrecGraph* g = nullptr;
  for (auto& e : h->pgraphs)
    if (e.in == in && e.out == out && e.nr == nr) g = &e;
  if (!g) {
    // capture; if the capture or the instantiation fails, this (in, out, n_rhs)
    // keeps running uncaptured (an entry without a graph)
    const long long l0 = h->launches;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool captured = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (captured) {
      try {
        precond_apply(h, in, out, nr, s);
      } catch (...) {
        captured = false;
      }
      const cudaError_t ec = cudaStreamEndCapture(s, &graph);
      captured = captured && ec == cudaSuccess && graph != nullptr;
      if (captured) captured = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();                          // a failed capture leaves no sticky error
    const long long nl = h->launches - l0;
    h->launches = l0;
    h->pgraphs.push_back({in, out, nr, captured ? exec : nullptr, nl});
    g = &h->pgraphs.back();
  }
  if (!g->exec) {
    precond_apply(h, in, out, nr, s);
    return;
  }
  HZ_CU(cudaGraphLaunch(g->exec, s));
  h->launches += g->launches;
}

void clear_graphs(hz_handle* h) {
  for (auto& e : h->pgraphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  h->pgraphs.clear();
  h->pwarm.clear();
}

}  // namespace hz
