// Set-up of a grid level: PML tables, medium copies, slab partition, slab meshes
// with the added DD PML and frozen k, slab stencils and transmission
// coefficients.  Everything is computed by kernels on the device.
#include "hz_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace hz {

long long test_hook(const char* name) {
  const char* v = std::getenv(name);
  if (!v || !*v) return -1;
  char* end = nullptr;
  const long long x = std::strtoll(v, &end, 10);
  return (end && *end == 0) ? x : -1;
}

void* dmalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  // test hook: a request of at least HZ_TEST_ALLOC_LIMIT bytes fails as if
  // the device were out of memory (exercises the HZ_ENOMEM paths on the host)
  const long long limit = test_hook("HZ_TEST_ALLOC_LIMIT");
  if (limit >= 0 && (long long)bytes >= limit)
    throw Failure(HZ_ENOMEM, "cudaMalloc(" + std::to_string(bytes) +
                                 ") refused by HZ_TEST_ALLOC_LIMIT");
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Failure(HZ_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + ") failed: " +
                                 cudaGetErrorString(e));
  }
  return p;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

// alpha = 1 / (1 + i sigma / omega)  (definition below Eq. 40)
__device__ __forceinline__ c128 pml_alpha(double sigma, double omega) {
  double a = sigma / omega;
  double d = 1.0 / (1.0 + a * a);
  return mk(d, -a * d);
}

// Uniform axis of n_cells cells, w_out PML cells per side (Eq. 5):
// sigma = C d^2, d = distance beyond the interior box [w_out h, (n_cells-w_out) h].
__global__ void fine_axis_kernel(int N, int n_cells, int w_out, double h, double C,
                                 double omega, c128* a_node, c128* a_cell, double* h_cell,
                                 c64* a_node32, c64* a_cell32, c128* ia_node, c64* ia_node32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > N) return;
  double lo = w_out * h, hi = (n_cells - w_out) * h;
  if (i < N) {
    double x = (i + 1) * h;
    double d = fmax(0.0, fmax(lo - x, x - hi));
    c128 a = pml_alpha(C * d * d, omega);
    a_node[i] = a;
    a_node32[i] = ccast<float>(a);
    const c128 ia = mk(1.0, C * d * d / omega);   // 1/alpha, exactly
    ia_node[i] = ia;
    ia_node32[i] = ccast<float>(ia);
  }
  double x = (i + 0.5) * h;
  double d = fmax(0.0, fmax(lo - x, x - hi));
  c128 a = pml_alpha(C * d * d, omega);
  a_cell[i] = a;
  a_cell32[i] = ccast<float>(a);
  h_cell[i] = h;
}

// Slab x axis (Eqs. 9-10 with the reading that the added PML starts at the
// interface half point): core unknowns/cells copy the global tables; the
// m-th added unknown is at distance (m - 1/2) h_I, added cells at (m - 1) h_I.
__global__ void slab_axis_kernel(int W, int lo, int hi, int wl, const c128* g_anode,
                                 const c128* g_acell, const double* g_hcell, double s_dd,
                                 double c_pml, int w, double omega, c128* a_node, c128* a_cell,
                                 double* h_cell, c64* a_node32, c64* a_cell32) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > W) return;
  double hIl = g_hcell[lo], hIr = g_hcell[hi + 1];
  double Cl = s_dd * c_pml / ((w * hIl) * (w * hIl) * (w * hIl));
  double Cr = s_dd * c_pml / ((w * hIr) * (w * hIr) * (w * hIr));
  if (e < W) {
    int g = e - wl + lo;
    c128 a;
    if (g < lo) {
      double d = (lo - g - 0.5) * hIl;
      a = pml_alpha(Cl * d * d, omega);
    } else if (g > hi) {
      double d = (g - hi - 0.5) * hIr;
      a = pml_alpha(Cr * d * d, omega);
    } else {
      a = g_anode[g];
    }
    a_node[e] = a;
    a_node32[e] = ccast<float>(a);
  }
  int gc = e - wl + lo;
  c128 a;
  double hc;
  if (gc < lo) {
    double d = (lo - gc) * hIl;
    a = pml_alpha(Cl * d * d, omega);
    hc = hIl;
  } else if (gc > hi + 1) {
    double d = (gc - hi - 1) * hIr;
    a = pml_alpha(Cr * d * d, omega);
    hc = hIr;
  } else {
    a = g_acell[gc];
    hc = g_hcell[gc];
  }
  a_cell[e] = a;
  a_cell32[e] = ccast<float>(a);
  h_cell[e] = hc;
}

// Slab stencil of the 5-point operator (Eq. 40 x h^2) on the extended slab
// mesh, k frozen to the adjacent core column in the added PML (Eq. 10).
// Layout st[k][9][W], plane (dy+1)*3+(dx+1); couplings to Dirichlet nodes
// are zero.
template <typename R>
__global__ void slab_stencil_fd_kernel(int W, int wp, int ny, int lo, int hi, int wl, int nx,
                                       double h2w2, const double* m, const c128* sa_node,
                                       const c128* sa_cell, const c128* ay_node,
                                       const c128* ay_cell, const double* bx, const double* by,
                                       cplx<R>* st) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (e >= W || k >= ny) return;
  int g = min(max(e - wl + lo, lo), hi);
  double mm = m[(size_t)k * nx + g];
  c128 inv_a2 = cinv(ay_node[k]);
  c128 inv_a1 = cinv(sa_node[e]);
  c128 a1l = sa_cell[e], a1r = sa_cell[e + 1];
  c128 a2d = ay_cell[k], a2u = ay_cell[k + 1];
  // sponge: k^2 (1 + i beta)^2, frozen with k in the added columns (Eq. 10)
  const c128 sp = bx ? sponge_s(bx[g] + by[k]) : mk(1.0, 0.0);
  c128 diag = inv_a2 * (a1l + a1r) + inv_a1 * (a2d + a2u) -
              (h2w2 * mm) * (sp * (inv_a1 * inv_a2));
  c128 z = mk(0.0, 0.0);
  c128 v[9];
  for (int q = 0; q < 9; ++q) v[q] = z;
  v[4] = diag;
  v[3] = (e > 0) ? -(inv_a2 * a1l) : z;
  v[5] = (e < W - 1) ? -(inv_a2 * a1r) : z;
  v[1] = (k > 0) ? -(inv_a1 * a2d) : z;
  v[7] = (k < ny - 1) ? -(inv_a1 * a2u) : z;
  cplx<R>* out = st + (size_t)k * 9 * wp;
  for (int q = 0; q < 9; ++q) out[q * wp + e] = ccast<R>(v[q]);
}

// Transmission coefficients of Eqs. 19-20 for the 5-point operator (only the
// dy = 0 coupling is non-zero): the global coupling between columns x and
// x+1 at row k is A_{(k,x),(k,x+1)} = -alpha_{1,x+1/2} / alpha_{2,k}.
//   inj[0][k] = +A_{beta,beta+1}      (row beta   of T B, multiplies B[1])
//   inj[1][k] = -A_{beta+1,beta}      (row beta+1 of T B, multiplies B[0])
//   inj[2][k] = -A_{bt,bt+1}          (row bt     of T~ B, multiplies B[1])
//   inj[3][k] = +A_{bt+1,bt}          (row bt+1   of T~ B, multiplies B[0])
// with beta = beta_{j-1}, bt = tilde-beta_j.  Stored [4][ny][3] (dy = -1,0,1).
template <typename R>
__global__ void inj_fd_kernel(int ny, int beta, int bt, const c128* ax_cell,
                              const c128* ay_node, cplx<R>* inj) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ny) return;
  c128 inv_a2 = cinv(ay_node[k]);
  c128 z = mk(0.0, 0.0);
  c128 af = (beta >= 0) ? -(inv_a2 * ax_cell[beta + 1]) : z;
  c128 ab = (bt >= 0) ? -(inv_a2 * ax_cell[bt + 1]) : z;
  c128 vals[4] = {af, -af, -ab, ab};
  for (int q = 0; q < 4; ++q) {
    cplx<R>* o = inj + ((size_t)q * ny + k) * 3;
    o[0] = ccast<R>(z);
    o[1] = ccast<R>(vals[q]);
    o[2] = ccast<R>(z);
  }
}

// Same for a stored 9-point operator (planes st[(dy+1)*3+(dx+1)][y][x]).
template <typename R>
__global__ void inj_fe_kernel(int ny, int nx, int beta, int bt, const c128* st, cplx<R>* inj) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ny) return;
  size_t plane = (size_t)ny * nx;
  for (int d = 0; d < 3; ++d) {
    int dy = d - 1;
    c128 z = mk(0.0, 0.0);
    c128 f0 = z, f1 = z, b0 = z, b1 = z;
    if (beta >= 0) {
      f0 = st[(size_t)(d * 3 + 2) * plane + (size_t)k * nx + beta];         // A_{(k,b),(k+dy,b+1)}
      f1 = -st[(size_t)(d * 3 + 0) * plane + (size_t)k * nx + beta + 1];    // -A_{(k,b+1),(k+dy,b)}
    }
    if (bt >= 0) {
      b0 = -st[(size_t)(d * 3 + 2) * plane + (size_t)k * nx + bt];
      b1 = st[(size_t)(d * 3 + 0) * plane + (size_t)k * nx + bt + 1];
    }
    c128 vals[4] = {f0, f1, b0, b1};
    for (int q = 0; q < 4; ++q) inj[((size_t)q * ny + k) * 3 + d] = ccast<R>(vals[q]);
  }
}

__global__ void mean_inv_sqrt_kernel(const double* m, size_t n, double* partial) {
  __shared__ double sh[256];
  double acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    acc += 1.0 / sqrt(m[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

double mean_velocity(const double* m_dev, size_t n, cudaStream_t s) {
  const int blocks = 304;
  double* part = (double*)dmalloc(blocks * sizeof(double));
  mean_inv_sqrt_kernel<<<blocks, 256, 0, s>>>(m_dev, n, part);
  std::vector<double> hp(blocks);
  cudaError_t e = cudaMemcpyAsync(hp.data(), part, blocks * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(part);
  if (e != cudaSuccess) throw Failure(HZ_ECUDA, std::string("mean velocity: ") + cudaGetErrorString(e));
  double acc = 0;
  for (double v : hp) acc += v;
  return acc / (double)n;
}

static void alloc_axis(AxisTables& a, int N) {
  a.N = N;
  a.a_node = (c128*)dmalloc(sizeof(c128) * N);
  a.a_cell = (c128*)dmalloc(sizeof(c128) * (N + 1));
  a.h_cell = (double*)dmalloc(sizeof(double) * (N + 1));
  a.a_node32 = (c64*)dmalloc(sizeof(c64) * N);
  a.a_cell32 = (c64*)dmalloc(sizeof(c64) * (N + 1));
}

static void free_axis(AxisTables& a) {
  dfree(a.a_node); dfree(a.a_cell); dfree(a.h_cell); dfree(a.a_node32); dfree(a.a_cell32);
  dfree(a.ia_node); dfree(a.ia_node32);
  dfree(a.beta); dfree(a.beta32);
  a = AxisTables{};
}

__global__ void to_float_kernel(const double* a, float* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

SegmentLayout segment_layout(int ny, int segments, int max_auto) {
  if (ny < 3) throw Failure(HZ_EINVAL, "a slab needs at least 3 rows");
  SegmentLayout L;
  L.mid = (ny - 1) / 2;
  const int ntop = L.mid, nbot = ny - 1 - L.mid;
  int P = segments;
  if (P <= 0) P = std::min(2 * (int)std::lround(std::pow((double)ny, 2.0 / 3.0)), std::max(2, max_auto));
  P = std::max(2, std::min(P, ny - 1));
  int S0 = (P * ntop + ny / 2) / (ny - 1);      // segments in proportion to the chain lengths
  S0 = std::max(1, std::min(S0, std::min(P - 1, ntop)));
  const int S1 = std::min(P - S0, nbot);
  P = S0 + S1;
  L.P = P;
  L.S0 = S0;
  L.seg.assign(P, int4{0, 0, 0, 0});
  for (int q = 0; q < S0; ++q) {
    const int a0 = (int)((long long)ntop * q / S0), a1 = (int)((long long)ntop * (q + 1) / S0);
    L.seg[q] = int4{a0, a1 - a0, +1, 0};
  }
  for (int q = 0; q < S1; ++q) {
    const int a0 = (int)((long long)nbot * q / S1), a1 = (int)((long long)nbot * (q + 1) / S1);
    L.seg[S0 + q] = int4{ny - 1 - a0, a1 - a0, -1, 0};
  }
  // groups: about sqrt(segments) per half, sizes differing by at most one
  auto make_groups = [&](int s_first, int nh, int half) {
    const int ng = std::max(1, std::min(nh, (int)std::lround(std::sqrt((double)nh))));
    for (int c = 0; c < ng; ++c) {
      const int a0 = s_first + nh * c / ng, a1 = s_first + nh * (c + 1) / ng;
      const int gi = (int)L.grp.size();
      L.grp.push_back(int4{a0, a1 - 1, half, c});
      for (int q = a0; q < a1; ++q) L.seg[q].w = gi;
    }
    return ng;
  };
  L.G0 = make_groups(0, S0, 0);
  L.NG = L.G0 + make_groups(S0, S1, 1);
  return L;
}

// n_int[l]: interior cells along x, y, z (z only when dim3d).
void build_level_fd(hz_handle* h, Level& L, const int* n_int, int w_out, double hh,
                    const double* m_dev, bool dim3d, cudaStream_t s) {
  L.dim3d = dim3d;
  L.nx = n_int[0] + 2 * w_out - 1;
  L.ny = n_int[1] + 2 * w_out - 1;
  L.nz = dim3d ? n_int[2] + 2 * w_out - 1 : 1;
  L.h = hh;
  L.fe = false;
  const bool sponge = h->p.boundary == HZ_BOUNDARY_SPONGE;
  // the outer layers: PML (Eq. 5), or a sponge (no PML; alpha = 1)
  double C = (w_out > 0 && !sponge) ? h->p.s_pml_out * h->c_pml / std::pow(w_out * hh, 3) : 0.0;
  // sponge: beta = beta_max (d / (w_out h))^2 per axis, beta_max from the
  // one-way damping exp(-k beta_max w_out h / 3) at k = omega / c_pml
  const double bmax = sponge ? 3.0 * std::log(1.0 / h->p.sponge_damping) /
                                   (h->p.omega / h->c_pml * w_out * hh)
                             : 0.0;
  AxisTables* axes[3] = {&L.ax, &L.ay, &L.az};
  for (int l = 0; l < (dim3d ? 3 : 2); ++l) {
    AxisTables* a = axes[l];
    const int n_cells = n_int[l] + 2 * w_out;
    const int N = n_cells - 1;
    alloc_axis(*a, N);
    a->ia_node = (c128*)dmalloc(sizeof(c128) * N);
    a->ia_node32 = (c64*)dmalloc(sizeof(c64) * N);
    fine_axis_kernel<<<cdiv(N + 1, 256), 256, 0, s>>>(
        N, n_cells, w_out, hh, C, h->p.omega, a->a_node, a->a_cell, a->h_cell, a->a_node32,
        a->a_cell32, a->ia_node, a->ia_node32);
    HZ_CU(cudaGetLastError());
    std::vector<double> beta(N, 0.0);
    if (sponge) {
      const double lo = w_out * hh, hi = (n_cells - w_out) * hh;
      std::vector<float> b32(N);
      for (int i = 0; i < N; ++i) {
        const double x = (i + 1) * hh;
        const double d = std::max(0.0, std::max(lo - x, x - hi)) / (w_out * hh);
        beta[i] = bmax * d * d;
        b32[i] = (float)beta[i];
      }
      a->beta = (double*)dmalloc(sizeof(double) * N);
      a->beta32 = (float*)dmalloc(sizeof(float) * N);
      HZ_CU(cudaMemcpyAsync(a->beta, beta.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
      HZ_CU(cudaMemcpyAsync(a->beta32, b32.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s));
    }
    // PML- and sponge-free interior (the operator's coefficients are real
    // there): the longest run of unknowns with 1/alpha = 1 at the node and
    // alpha = 1 at both adjacent cells, read back from the tables just built,
    // and beta = 0
    std::vector<c128> ia(N), ac(N + 1);
    HZ_CU(cudaMemcpyAsync(ia.data(), a->ia_node, sizeof(c128) * N, cudaMemcpyDeviceToHost, s));
    HZ_CU(cudaMemcpyAsync(ac.data(), a->a_cell, sizeof(c128) * (N + 1), cudaMemcpyDeviceToHost,
                          s));
    HZ_CU(cudaStreamSynchronize(s));
    auto one = [](const c128& v) { return v.re == 1.0 && v.im == 0.0; };
    int best_lo = 1, best_hi = 0, run = -1;
    for (int i = 0; i <= N; ++i) {
      const bool ok = i < N && one(ia[i]) && one(ac[i]) && one(ac[i + 1]) && beta[i] == 0.0;
      if (ok && run < 0) run = i;
      if (!ok && run >= 0) {
        if (i - 1 - run > best_hi - best_lo) { best_lo = run; best_hi = i - 1; }
        run = -1;
      }
    }
    a->in_lo = best_lo;
    a->in_hi = best_hi;
  }
  size_t nn = L.size();
  if (!L.m) L.m = (double*)dmalloc(sizeof(double) * nn);
  if (!L.m32) L.m32 = (float*)dmalloc(sizeof(float) * nn);
  HZ_CU(cudaMemcpyAsync(L.m, m_dev, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  to_float_kernel<<<cdiv(nn, 256), 256, 0, s>>>(L.m, L.m32, nn);
  HZ_CU(cudaGetLastError());
}

// Partition (Eq. 17): beta_0 = -1, beta_J = N-1, first N mod J slabs one wider.
void partition(Level& L) {
  int N = L.nx, J = L.J;
  L.beta.assign(J + 1, 0);
  L.beta[0] = -1;
  for (int j = 0; j < J; ++j) L.beta[j + 1] = L.beta[j] + N / J + (j < N % J ? 1 : 0);
  L.beta_t = L.beta;
  for (int j = 1; j < J; ++j) L.beta_t[j] = L.beta[j] - 1;
}

// Slab j of the partition: core columns, added PML columns (Eq. 9) and the
// slab x axis with the DD PML (Eqs. 9-10).
void slab_geometry(hz_handle* h, Level& L, Slab& S, int j, cudaStream_t s) {
  S.j = j;
  S.lo = L.beta_t[j - 1] + 1;
  S.hi = L.beta[j];
  S.wl = (j > 1) ? L.w : 0;
  S.wr = (j < L.J) ? L.w : 0;
  S.W = S.hi - S.lo + 1 + S.wl + S.wr;
  alloc_axis(S.ax, S.W);
  slab_axis_kernel<<<cdiv(S.W + 1, 128), 128, 0, s>>>(
      S.W, S.lo, S.hi, S.wl, L.ax.a_node, L.ax.a_cell, L.ax.h_cell, h->p.s_pml_dd, h->c_pml,
      L.w, h->p.omega, S.ax.a_node, S.ax.a_cell, S.ax.h_cell, S.ax.a_node32, S.ax.a_cell32);
  HZ_CU(cudaGetLastError());
}

template <typename R>
static void build_slabs_t(hz_handle* h, Level& L, cudaStream_t s) {
  partition(L);
  L.slabs.assign(L.J + 1, Slab{});
  int maxW = 0;
  for (int j = 1; j <= L.J; ++j) {
    Slab& S = L.slabs[j];
    slab_geometry(h, L, S, j, s);
    maxW = std::max(maxW, S.W);
    // plane stride padded so that every plane row starts on a 16-byte boundary
    // row stride = 4 (mod 8): rows start on 16-byte boundaries and the eight
    // rows a warp reads in one substitution step fall on disjoint bank groups
    S.wp = S.W + ((4 - S.W % 8) + 8) % 8;
    S.st = dmalloc(sizeof(cplx<R>) * (size_t)L.ny * 9 * S.wp);
    HZ_CU(cudaMemsetAsync(S.st, 0, sizeof(cplx<R>) * (size_t)L.ny * 9 * S.wp, s));
    S.inj = dmalloc(sizeof(cplx<R>) * 4 * (size_t)L.ny * 3);
    int beta = (j > 1) ? L.beta[j - 1] : -1;
    int bt = (j < L.J) ? L.beta_t[j] : -1;
    if (!L.fe) {
      dim3 grid(cdiv(S.W, 128), L.ny);
      double h2w2 = L.h * L.h * h->p.omega * h->p.omega;
      slab_stencil_fd_kernel<R><<<grid, 128, 0, s>>>(S.W, S.wp, L.ny, S.lo, S.hi, S.wl, L.nx, h2w2,
                                                     L.m, S.ax.a_node, S.ax.a_cell, L.ay.a_node,
                                                     L.ay.a_cell, L.ax.beta, L.ay.beta,
                                                     (cplx<R>*)S.st);
      inj_fd_kernel<R><<<cdiv(L.ny, 128), 128, 0, s>>>(L.ny, beta, bt, L.ax.a_cell, L.ay.a_node,
                                                       (cplx<R>*)S.inj);
    } else {
      slab_stencil_fe<R>(h, L, S, s);
      inj_fe_kernel<R><<<cdiv(L.ny, 128), 128, 0, s>>>(L.ny, L.nx, beta, bt, L.st128,
                                                       (cplx<R>*)S.inj);
    }
    HZ_CU(cudaGetLastError());
    // factor storage: W*W elements rounded up to a 16-byte multiple per block row
    size_t per = (size_t)S.W * S.W;
    size_t elems16 = 16 / sizeof(cplx<R>);
    if (elems16 < 1) elems16 = 1;
    S.gstride = (per + elems16 - 1) / elems16 * elems16;
    S.G = dmalloc(sizeof(cplx<R>) * S.gstride * L.ny);
    S.mstride = (size_t)S.W * S.wp;
    S.F = dmalloc(sizeof(cplx<R>) * S.mstride * L.ny);
    S.E = dmalloc(sizeof(cplx<R>) * S.mstride * L.ny);
    HZ_CU(cudaMemsetAsync(S.F, 0, sizeof(cplx<R>) * S.mstride * L.ny, s));   // zero padding
    HZ_CU(cudaMemsetAsync(S.E, 0, sizeof(cplx<R>) * S.mstride * L.ny, s));
    S.Y = dmalloc(sizeof(cplx<R>) * (size_t)h->p.max_rhs * L.ny * S.wp);
  }
  // Twisted elimination: chains from rows 0 and ny-1 meet at row mid.  Each
  // chain is cut into P/2 segments of L ~ ny / P rows for the parallel
  // substitution, and the segments of a half into about sqrt(P/2) groups for
  // the two-level carries.  Sequential steps of a solve per half: ~4 L in
  // the segment passes plus ~4 sqrt(P/2) in the carries; the minimum lies at
  // P/2 ~ ny^(2/3).  Automatic P is that, capped so that every segment pass
  // (one CTA per segment) is one wave: twice the SM count in complex64 (two
  // segment CTAs with 2-stage pipelines share an SM), the SM count in
  // complex128 (one CTA with its full pipeline per SM).
  const int per_sm = (h->p.precision == HZ_MIXED) ? 2 : 1;
  SegmentLayout lay = segment_layout(L.ny, h->p.segments, std::max(2, per_sm * h->sms));
  L.mid = lay.mid;
  L.P = lay.P;
  L.S0 = lay.S0;
  L.G0 = lay.G0;
  L.NG = lay.NG;
  L.seg = lay.seg;
  L.grp = lay.grp;
  const int P = L.P;
  L.seg_dev = (int4*)dmalloc(sizeof(int4) * (P + L.NG));
  L.grp_dev = L.seg_dev + P;
  HZ_CU(cudaMemcpyAsync(L.seg_dev, L.seg.data(), sizeof(int4) * P, cudaMemcpyHostToDevice, s));
  HZ_CU(cudaMemcpyAsync(L.grp_dev, L.grp.data(), sizeof(int4) * L.NG, cudaMemcpyHostToDevice, s));
  for (int j = 1; j <= L.J; ++j) {
    Slab& S = L.slabs[j];
    const size_t pb = sizeof(cplx<R>) * S.mstride * P;
    S.Phi = dmalloc(pb);
    S.Psi = dmalloc(pb);
    S.PhiP = dmalloc(pb);
    S.PsiP = dmalloc(pb);
    S.carry_f = dmalloc(sizeof(cplx<R>) * (size_t)(P + L.NG) * h->p.max_rhs * S.wp);
    S.carry_b = dmalloc(sizeof(cplx<R>) * (size_t)(P + 1 + L.NG) * h->p.max_rhs * S.wp);
    HZ_CU(cudaMemsetAsync(S.Phi, 0, pb, s));      // zero padding
    HZ_CU(cudaMemsetAsync(S.Psi, 0, pb, s));
    HZ_CU(cudaMemsetAsync(S.PhiP, 0, pb, s));
    HZ_CU(cudaMemsetAsync(S.PsiP, 0, pb, s));
  }
  HZ_CU(cudaStreamSynchronize(s));
}

void build_slabs(hz_handle* h, Level& L, cudaStream_t s) {
  if (L.dim3d) {
    partition(L);
    if (h->p.precision == HZ_MIXED)
      build_slabs3d<float>(h, L, s);
    else
      build_slabs3d<double>(h, L, s);
    return;
  }
  if (h->p.precision == HZ_MIXED)
    build_slabs_t<float>(h, L, s);
  else
    build_slabs_t<double>(h, L, s);
}

void free_level(Level& L) {
  for (Slab& S : L.slabs) {
    free_axis(S.ax);
    dfree(S.st); dfree(S.G); dfree(S.F); dfree(S.E); dfree(S.Phi); dfree(S.Psi);
    dfree(S.PhiP); dfree(S.PsiP);
    dfree(S.inj); dfree(S.Y);
    dfree(S.carry_f); dfree(S.carry_b);
    dfree(S.st3); dfree(S.inj3); dfree(S.V); dfree(S.gpart); dfree(S.Gp); dfree(S.Vp);
  }
  L.slabs.clear();
  free_axis(L.ax);
  free_axis(L.ay);
  free_axis(L.az);
  dfree(L.m); dfree(L.m32); dfree(L.st128); dfree(L.st64); dfree(L.seg_dev);
  dfree(L.k2c); dfree(L.k2ci);
  for (int l = 0; l < 3; ++l) {
    dfree(L.ifp[l]); dfree(L.refined[l]); dfree(L.q0[l]); dfree(L.q1[l]);
  }
  dfree(L.fac_desc); dfree(L.fac_sync);
  dfree(L.f3_S); dfree(L.f3_C); dfree(L.f3_R); dfree(L.f3_piv); dfree(L.f3_pack); dfree(L.f3_desc);
  L = Level{};
}

}  // namespace hz
