// Slab factorisation and slab solves (the subdomain solves of SubdomSolve,
// Table 2; the paper uses a sparse direct solver, Section 5).
//
// A^(j) is block tridiagonal along y with W x W blocks (one block row per
// grid row k): D_k couples row k to itself, C_k to row k-1, B_k to row k+1
// (taken from the slab stencil st[k][9][wp], plane (dy+1)*3 + (dx+1)).
// Block LU:
//   S_0 = D_0,  S_k = D_k - C_k S_{k-1}^{-1} B_{k-1},  G_k = S_k^{-1} (stored).
// Solve A^(j) x = f:
//   forward   y_k = G_k (f_k - C_k y_{k-1})
//   backward  x_k = y_k - G_k (B_k x_{k+1})
// Parallel in y: the block rows are cut into P segments.  Both recurrences
// are affine, y_k = G_k f_k + F_k y_{k-1} with F_k = -G_k C_k and
// x_k = y_k + E_k x_{k+1} with E_k = -G_k B_k.  Per segment [a, b] the
// products Phi = F_b ... F_a and Psi = E_a ... E_b are formed at factor time;
// a solve runs each segment from a zero start (all segments in parallel),
// carries the segment end values through Phi / Psi (P short steps), and
// re-runs each segment from its true start value.
//
// Every block-row step reads its operands -- the factor block G_k, the
// coupling row C_k or B_k and the right-hand-side / forward row -- through
// one stage of a shared-memory pipeline filled by TMA bulk copies
// (cp.async.bulk + mbarrier); the step itself touches only shared memory and
// registers.
#include "hz_internal.h"

#include <algorithm>
#include <cmath>

namespace hz {

// ----------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy accesses (shared and global)
// before later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
// Same for shared memory only: issued before a TMA copy overwrites a stage
// that the block has just read with ordinary loads (a warp may pass the block
// barrier with such loads still in flight).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s, raises the device flag, returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer() - t0 > 2000000000ull) {
      atomicExch(flag, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

constexpr int kThreads = 512;
constexpr int kTPR = 4;                 // threads cooperating on one row of a GEMV
constexpr int kGroups = kThreads / kTPR;
constexpr int kNRMax = 8;               // right-hand sides per launch

// --------------------------------------------------------------- factorisation
struct FactorDesc {
  int W, wp, ny;
  const void* st;
  void* G;
  size_t gstride;
};

// One CTA per slab, sequential over block rows.  Each S_k is inverted by
// Gauss-Jordan elimination with partial pivoting; pivot rows are marked, not
// moved, and the permutations are applied when G_k is written:
// G_k[p][piv[q]] = S[piv[p]][q].  With colmod = column p of S except
// colmod[r] = S[r][p] - 1, and rowmod = row r of S scaled by inv = 1/S[r][p]
// except rowmod[p] = inv + 1, one elimination step (pivot row included) is the
// rank-1 update S -= colmod rowmod^T.  The steps are blocked by panels of BW
// columns: one warp eliminates the panel's BW pivots on the panel columns only
// (shuffles, no block barrier), the pivot rows' other columns follow from the
// short recurrence rowmod_t = (S[r_t] - sum_{s<t} colmod_s[r_t] rowmod_s) inv_t,
// and all threads apply the delayed rank-BW update S -= Cm^T R in 4 x TC
// register tiles.  Three block barriers per panel.
__device__ __forceinline__ cplx<float> crcp(cplx<float> a) {
  const float d = __frcp_rn(a.re * a.re + a.im * a.im);
  return mk(a.re * d, -a.im * d);
}
__device__ __forceinline__ cplx<double> crcp(cplx<double> a) {
  const double d = __drcp_rn(a.re * a.re + a.im * a.im);
  return mk(a.re * d, -a.im * d);
}

template <typename R>
struct FactorPanel { static constexpr int BW = 8; };
template <>
struct FactorPanel<double> { static constexpr int BW = 4; };

// One warp eliminates pivots p0 .. p0+bw-1 on the panel columns p0 .. p0+bw-1
// (rows lane + 32 m, m < MR, in registers) and records colmod (Cm), the pivot
// inverses and rows.
template <typename R, int BW, int MR>
__device__ __forceinline__ void panel_elim(cplx<R>* S, cplx<R>* Cm, cplx<R>* pinv, int* prow,
                                           int* piv, int* used, int W, int p0, int bw, int lane) {
  const cplx<R> zero = mk<R>(0, 0);
  cplx<R> P[MR][BW];
  bool usd[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = lane + 32 * m;
    usd[m] = (i < W) ? (used[i] != 0) : true;
#pragma unroll
    for (int c = 0; c < BW; ++c) P[m][c] = (i < W && c < bw) ? S[i * W + p0 + c] : zero;
  }
#pragma unroll
  for (int t = 0; t < BW; ++t) {
    if (t < bw) {
      float lbv = -1.0f;
      int lbi = 1 << 30;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        if (!usd[m]) {
          const float v = (float)cabs2(P[m][t]);
          if (v > lbv) { lbv = v; lbi = lane + 32 * m; }
        }
      }
      const unsigned key = lbv >= 0.0f ? __float_as_uint(lbv) : 0u;
      const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
      const unsigned win = __ballot_sync(0xffffffffu, key == kmax && lbi < (1 << 30));
      const int r = __shfl_sync(0xffffffffu, lbi, __ffs(win) - 1);
      const int rl = r & 31, rm = r >> 5;
      cplx<R> prw[BW];
#pragma unroll
      for (int c = 0; c < BW; ++c) {
        cplx<R> x = P[0][c];
#pragma unroll
        for (int m = 1; m < MR; ++m)
          if (rm == m) x = P[m][c];
        prw[c].re = __shfl_sync(0xffffffffu, x.re, rl);
        prw[c].im = __shfl_sync(0xffffffffu, x.im, rl);
      }
      const cplx<R> inv = crcp(prw[t]);
      cplx<R> rowm[BW];
#pragma unroll
      for (int c = 0; c < BW; ++c)
        rowm[c] = (c == t) ? mk<R>(inv.re + (R)1, inv.im) : prw[c] * inv;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int i = lane + 32 * m;
        cplx<R> cm = P[m][t];
        if (i == r) { cm.re -= (R)1; usd[m] = true; }
        if (i < W) Cm[t * W + i] = cm;
#pragma unroll
        for (int c = 0; c < BW; ++c) {
          P[m][c].re -= cm.re * rowm[c].re - cm.im * rowm[c].im;
          P[m][c].im -= cm.re * rowm[c].im + cm.im * rowm[c].re;
        }
      }
      if (lane == 0) {
        pinv[t] = inv;
        prow[t] = r;
        piv[p0 + t] = r;
        used[r] = 1;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = lane + 32 * m;
#pragma unroll
    for (int c = 0; c < BW; ++c)
      if (i < W && c < bw) S[i * W + p0 + c] = P[m][c];
  }
}

template <typename R, int TC>
__global__ void __launch_bounds__(kThreads) slab_factor_kernel(const FactorDesc* descs) {
  constexpr int BW = FactorPanel<R>::BW;
  constexpr int TR = 4;
  const FactorDesc d = descs[blockIdx.x];
  const int W = d.W, wp = d.wp, ny = d.ny, tid = threadIdx.x;
  const int WW = W * W;
  const int lane = tid & 31, warp = tid >> 5;
  const int ntc = (W + TC - 1) / TC;             // tiles per row of S
  const int ntr = (W + TR - 1) / TR;
  const bool tile_owner = tid < ntr * ntc;
  const int ti0 = tile_owner ? (tid / ntc) * TR : 0;
  const int tj0 = tile_owner ? (tid % ntc) * TC : 0;
  const cplx<R>* st = (const cplx<R>*)d.st;
  cplx<R>* G = (cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* S = (cplx<R>*)smem_raw;               // W*W
  cplx<R>* Gl = S + WW;                          // W*W: G_{k-1}, natural order
  cplx<R>* Cm = Gl + WW;                         // BW x W  (colmod of the panel's pivots)
  cplx<R>* Rm = Cm + BW * W;                     // BW x W  (rowmod on the other columns)
  cplx<R>* cC = Rm + BW * W;                     // C_k (3 x W)
  cplx<R>* cD = cC + 3 * W;                      // D_k (3 x W)
  cplx<R>* cB = cD + 3 * W;                      // B_{k-1} (3 x W)
  cplx<R>* pinv = cB + 3 * W;                    // BW
  int* prow = (int*)(pinv + BW);                 // BW
  int* piv = prow + BW;                          // W
  int* ipiv = piv + W;                           // W
  int* used = ipiv + W;                          // W
  const cplx<R> zero = mk<R>(0, 0);

  for (int k = 0; k < ny; ++k) {
    const cplx<R>* stk = st + (size_t)k * 9 * wp;
    for (int t = tid; t < 3 * W; t += kThreads) {     // stage the couplings
      const int q = t / W, e = t - q * W;
      cC[t] = stk[q * wp + e];
      cD[t] = stk[(3 + q) * wp + e];
      cB[t] = (k > 0) ? st[(size_t)(k - 1) * 9 * wp + (6 + q) * wp + e] : zero;
    }
    for (int t = tid; t < W; t += kThreads) used[t] = 0;
    __syncthreads();
    // S_k = D_k - C_k G_{k-1} B_{k-1} (natural order, shared memory)
    if (k > 0) {
      for (int e = tid; e < WW; e += kThreads) {      // Cm-area is free: X = G B into S
        const int i = e / W, j = e - i * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int c = j - dx;
          if (c >= 0 && c < W) cfma(acc, Gl[i * W + c], cB[(dx + 1) * W + c]);
        }
        S[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < WW; e += kThreads) {      // Gl = D - C X
        const int i = e / W, j = e - i * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int rr = i + dx;
          if (rr >= 0 && rr < W) cfma(acc, cC[(dx + 1) * W + i], S[rr * W + j]);
        }
        cplx<R> v = -acc;
        const int dd = j - i;
        if (dd >= -1 && dd <= 1) v = v + cD[(dd + 1) * W + i];
        Gl[e] = v;
      }
      __syncthreads();
      for (int e = tid; e < WW; e += kThreads) S[e] = Gl[e];
    } else {
      for (int e = tid; e < WW; e += kThreads) {
        const int i = e / W, j = e - i * W;
        const int dd = j - i;
        S[e] = (dd >= -1 && dd <= 1) ? cD[(dd + 1) * W + i] : zero;
      }
    }
    __syncthreads();

    for (int p0 = 0; p0 < W; p0 += BW) {
      const int bw = min(BW, W - p0);
      // (1) one warp eliminates the panel's pivots on the panel columns
      if (warp == 0) {
        const int MR = (W + 31) >> 5;
        if (bw == BW) {
          if (MR == 1) panel_elim<R, BW, 1>(S, Cm, pinv, prow, piv, used, W, p0, bw, lane);
          else if (MR == 2) panel_elim<R, BW, 2>(S, Cm, pinv, prow, piv, used, W, p0, bw, lane);
          else if (MR == 3) panel_elim<R, BW, 3>(S, Cm, pinv, prow, piv, used, W, p0, bw, lane);
          else panel_elim<R, BW, 4>(S, Cm, pinv, prow, piv, used, W, p0, bw, lane);
        } else {
          panel_elim<R, BW, 4>(S, Cm, pinv, prow, piv, used, W, p0, bw, lane);
        }
      }
      __syncthreads();
      // (2) rowmod of the panel's pivots on the other columns
      for (int j = tid; j < W; j += kThreads) {
        if (j >= p0 && j < p0 + bw) continue;
        cplx<R> rw[BW];
#pragma unroll
        for (int t = 0; t < BW; ++t) {
          if (t >= bw) break;
          const int r = prow[t];
          cplx<R> acc = S[r * W + j];
#pragma unroll
          for (int q = 0; q < t; ++q) {
            const cplx<R> c = Cm[q * W + r];
            acc.re -= c.re * rw[q].re - c.im * rw[q].im;
            acc.im -= c.re * rw[q].im + c.im * rw[q].re;
          }
          rw[t] = acc * pinv[t];
          Rm[t * W + j] = rw[t];
        }
      }
      __syncthreads();
      // (3) delayed rank-bw update of the other columns, 4 x TC tiles
      if (tile_owner) {
        cplx<R> acc[TR][TC];
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
          for (int b = 0; b < TC; ++b) {
            const int i = ti0 + a, j = tj0 + b;
            acc[a][b] = (i < W && j < W) ? S[i * W + j] : zero;
          }
#pragma unroll
        for (int t = 0; t < BW; ++t) {
          if (t >= bw) break;
          cplx<R> cv[TR], rv[TC];
#pragma unroll
          for (int a = 0; a < TR; ++a) cv[a] = (ti0 + a < W) ? Cm[t * W + ti0 + a] : zero;
#pragma unroll
          for (int b = 0; b < TC; ++b) {
            const int j = tj0 + b;
            rv[b] = (j < W && (j < p0 || j >= p0 + bw)) ? Rm[t * W + j] : zero;
          }
#pragma unroll
          for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) {
              acc[a][b].re -= cv[a].re * rv[b].re - cv[a].im * rv[b].im;
              acc[a][b].im -= cv[a].re * rv[b].im + cv[a].im * rv[b].re;
            }
        }
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
          for (int b = 0; b < TC; ++b) {
            const int i = ti0 + a, j = tj0 + b;
            if (i < W && j < W && (j < p0 || j >= p0 + bw)) S[i * W + j] = acc[a][b];
          }
      }
      __syncthreads();
    }
    for (int q = tid; q < W; q += kThreads) ipiv[piv[q]] = q;
    __syncthreads();
    cplx<R>* Gk = G + (size_t)k * d.gstride;
    for (int e = tid; e < WW; e += kThreads) {
      const int i = e / W, j = e - i * W;
      const cplx<R> v = S[piv[i] * W + ipiv[j]];
      Gk[e] = v;
      Gl[e] = v;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ segment products
struct ProdDesc {
  int W, wp, k0, k1, backward;
  const void* st;
  const void* G;
  size_t gstride;
  void* out;
};

// forward:  M <- F_k M for k = k0..k1-1, F_k = -G_k C_k   (M = F_{k1-1} ... F_{k0})
// backward: M <- E_k M for k = k1-1..k0, E_k = -G_k B_k   (M = E_{k0} ... E_{k1-1})
template <typename R>
__global__ void __launch_bounds__(kThreads) segment_product_kernel(const ProdDesc* descs) {
  const ProdDesc d = descs[blockIdx.x];
  const int W = d.W, wp = d.wp, tid = threadIdx.x;
  const int ty = tid >> 2, tx = tid & 3;
  const cplx<R>* st = (const cplx<R>*)d.st;
  const cplx<R>* G = (const cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* M = (cplx<R>*)smem_raw;
  cplx<R>* T = M + W * W;
  const cplx<R> zero = mk<R>(0, 0);
  for (int i = tid; i < W * W; i += kThreads) M[i] = zero;
  __syncthreads();
  for (int i = tid; i < W; i += kThreads) M[i * W + i] = mk<R>(1, 0);
  __syncthreads();
  const int n = d.k1 - d.k0;
  const int plane = d.backward ? 6 : 0;   // B_k (dy=+1) or C_k (dy=-1)
  for (int s = 0; s < n; ++s) {
    const int k = d.backward ? d.k1 - 1 - s : d.k0 + s;
    const cplx<R>* stk = st + (size_t)k * 9 * wp;
    for (int i = ty; i < W; i += kGroups)          // T = coupling_k M
      for (int c = tx; c < W; c += kTPR) {
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          int e = i + dx;
          if (e >= 0 && e < W) cfma(acc, stk[(plane + dx + 1) * wp + i], M[e * W + c]);
        }
        T[i * W + c] = acc;
      }
    __syncthreads();
    const cplx<R>* Gk = G + (size_t)k * d.gstride;
    for (int i = ty; i < W; i += kGroups)          // M = -G_k T
      for (int c = tx; c < W; c += kTPR) {
        cplx<R> acc = zero;
        for (int j = 0; j < W; ++j) cfma(acc, Gk[i * W + j], T[j * W + c]);
        M[i * W + c] = -acc;
      }
    __syncthreads();
  }
  cplx<R>* out = (cplx<R>*)d.out;
  for (int i = tid; i < W * W; i += kThreads) out[i] = M[i];
}

// ------------------------------------------------------------------ solves
// Right-hand side of a slab solve: either a raw slab field, or the gather of
// global columns (ga, gb] plus the transmission injections of Table 2
// (lines 2-5) at the local columns ef (tau1, from B1) and eb (tau3, from B3).
template <typename R>
struct Rhs {
  const cplx<R>* raw;         // [n_rhs][ny][W] or null
  const cplx<R>* f;           // global field [n_rhs][ny][nx]
  int nx, lo, wl, ga, gb;
  const cplx<R>* B1;          // [2][n_rhs][ny]
  int ef;                     // local column of beta_{j-1} (tau1) or -1
  const cplx<R>* B3;
  int eb;                     // local column of tilde-beta_j (tau3) or -1
  const cplx<R>* inj;         // [4][ny][3]
};

// Epilogue of a slab solve (Table 2 lines 6-10).
template <typename R>
struct Out {
  cplx<R>* raw;               // [n_rhs][ny][W] or null
  cplx<R>* u;                 // global field [n_rhs][ny][nx]: columns (ua, ub] are stored
  int nx, lo, wl, ua, ub;     // (each sweep phase writes every column exactly once)
  cplx<R>* B2;                // [2][n_rhs][ny]: layers at local e2, e2+1 (tau2)
  int e2;
  cplx<R>* B4;                // layers at local e4, e4+1 (tau4)
  int e4;
};

template <typename R>
struct SolveArgs {
  int W, wp, ny, nr, P;
  const int* seg;
  const cplx<R>* st;          // [ny][9][wp]
  const cplx<R>* G;           // [ny][gstride]
  size_t gstride;
  int stages;
  cplx<R>* Y;                 // [ny][nr][wp]: gathered right-hand side, then forward rows
  cplx<R>* carry_f;           // [P][nr][wp]
  cplx<R>* carry_b;
  int* flag;
  Rhs<R> rhs;
  Out<R> out;
};

template <typename R>
__device__ __forceinline__ cplx<R> rhs_at(const Rhs<R>& q, int ny, int W, int nr, int r, int k,
                                          int e) {
  const cplx<R> zero = mk<R>(0, 0);
  if (q.raw) return q.raw[((size_t)r * ny + k) * W + e];
  cplx<R> v = zero;
  int g = e - q.wl + q.lo;
  if (g > q.ga && g <= q.gb) v = q.f[((size_t)r * ny + k) * q.nx + g];
  if (q.ef >= 0 && (e == q.ef || e == q.ef + 1)) {
    int s = e - q.ef;                          // 0: row beta uses B[1]; 1: row beta+1 uses B[0]
    const cplx<R>* c = q.inj + ((size_t)s * ny + k) * 3;
    const cplx<R>* B = q.B1 + ((size_t)(1 - s) * nr + r) * ny;
    for (int dy = -1; dy <= 1; ++dy) {
      int kk = k + dy;
      if (kk >= 0 && kk < ny) cfma(v, c[dy + 1], B[kk]);
    }
  }
  if (q.eb >= 0 && (e == q.eb || e == q.eb + 1)) {
    int s = e - q.eb;
    const cplx<R>* c = q.inj + ((size_t)(2 + s) * ny + k) * 3;
    const cplx<R>* B = q.B3 + ((size_t)(1 - s) * nr + r) * ny;
    for (int dy = -1; dy <= 1; ++dy) {
      int kk = k + dy;
      if (kk >= 0 && kk < ny) cfma(v, c[dy + 1], B[kk]);
    }
  }
  return v;
}

// Pipeline stage: [G_k (gstride) | coupling row (3 wp) | vector row (nr wp)].
template <typename R>
struct Pipe {
  uint64_t* bar;
  cplx<R>* buf;
  int stages;
  size_t stage_elems, gstride;
  int wp, nr;
  __device__ cplx<R>* slot(int i) const { return buf + (size_t)i * stage_elems; }
  // thread 0 only: fetch block row k (coupling plane 0 = C_k or 6 = B_k)
  __device__ void issue(int i, int k, const cplx<R>* G, const cplx<R>* st, int plane,
                        const cplx<R>* rows) const {
    const uint32_t gb = (uint32_t)(gstride * sizeof(cplx<R>));
    const uint32_t cb = (uint32_t)(3 * wp * sizeof(cplx<R>));
    const uint32_t vb = (uint32_t)((size_t)nr * wp * sizeof(cplx<R>));
    cplx<R>* dst = slot(i);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[i], gb + cb + vb);
    tma_load_1d(dst, G + (size_t)k * gstride, gb, &bar[i]);
    tma_load_1d(dst + gstride, st + (size_t)k * 9 * wp + plane * wp, cb, &bar[i]);
    tma_load_1d(dst + gstride + 3 * wp, rows + (size_t)k * nr * wp, vb, &bar[i]);
  }
};

// acc[r] = sum_j M[row][j] v[r][j] for r < nr; every thread of the block calls
// this with the same trip count (rows >= W contribute zeros) so that the
// shuffles stay warp-uniform.  Two partial sums shorten the FMA chain.
template <typename R, int NR>
__device__ __forceinline__ void gemv_rows(const cplx<R>* M, int ldm, const cplx<R>* v, int ldv,
                                          int W, int nr, int row, int lane, cplx<R> (&acc)[NR]) {
  cplx<R> a0[NR], a1[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { a0[r] = mk<R>(0, 0); a1[r] = mk<R>(0, 0); }
  const cplx<R>* Mr = M + (size_t)row * ldm;
  const int jend = row < W ? W : 0;
  int j = lane;
  for (; j + kTPR < jend; j += 2 * kTPR) {
    const cplx<R> m0 = Mr[j], m1 = Mr[j + kTPR];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) {
        cfma(a0[r], m0, v[r * ldv + j]);
        cfma(a1[r], m1, v[r * ldv + j + kTPR]);
      }
  }
  if (j < jend) {
    const cplx<R> m0 = Mr[j];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) cfma(a0[r], m0, v[r * ldv + j]);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    acc[r] = a0[r] + a1[r];
#pragma unroll
    for (int o = kTPR / 2; o > 0; o >>= 1) {
      acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, o);
      acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, o);
    }
  }
}

template <typename R>
__device__ __forceinline__ void init_pipe(Pipe<R>& pipe, unsigned char* smem, const SolveArgs<R>& a,
                                          int NR, cplx<R>** vbuf, cplx<R>** ybuf) {
  pipe.bar = (uint64_t*)smem;
  *vbuf = (cplx<R>*)(smem + 128);
  *ybuf = *vbuf + NR * a.wp;
  cplx<R>* b = *ybuf + NR * a.wp;
  pipe.buf = (cplx<R>*)(((uintptr_t)b + 127) & ~(uintptr_t)127);
  pipe.stages = a.stages;
  pipe.gstride = a.gstride;
  pipe.wp = a.wp;
  pipe.nr = a.nr;
  pipe.stage_elems = a.gstride + 3 * (size_t)a.wp + (size_t)a.nr * a.wp;
}

// SubdomSolve lines 1-5: the slab right-hand side (gather + transmission
// injection) into the rows Y[k][r][0..wp).  A kernel of its own, so that the
// TMA reads of these rows in the next launch see them.
template <typename R>
__global__ void slab_gather_kernel(SolveArgs<R> a) {
  const int rowlen = a.nr * a.wp;
  const size_t total = (size_t)a.ny * rowlen;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k = (int)(idx / rowlen), rem = (int)(idx - (size_t)k * rowlen);
  const int r = rem / a.wp, e = rem - r * a.wp;
  a.Y[idx] = (e < a.W) ? rhs_at<R>(a.rhs, a.ny, a.W, a.nr, r, k, e) : mk<R>(0, 0);
}

// Forward recurrence over one segment.
//   mode 0: zero start, store only the segment's last y into carry_f[p];
//   mode 1: start from carry_f[p-1] (segment 0: zero), store every y_k into
//           Y (over the right-hand side); if bwd1, then run the backward
//           recurrence over the segment from a zero start and store its first
//           x into carry_b[p].
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_fwd_kernel(SolveArgs<R> a, int mode, int bwd1) {
  const int p = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, ny = a.ny, nr = a.nr;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  const int k0 = a.seg[p], k1 = a.seg[p + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  Pipe<R> pipe;
  cplx<R>* vbuf;
  cplx<R>* ybuf;
  init_pipe<R>(pipe, smem_raw, a, NR, &vbuf, &ybuf);
  const cplx<R> zero = mk<R>(0, 0);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
  }
  for (int i = tid; i < NR * wp; i += nthr) {
    const int r = i / wp, e = i - r * wp;
    ybuf[i] = (mode == 1 && p > 0 && r < nr) ? a.carry_f[((size_t)(p - 1) * nr + r) * wp + e] : zero;
  }
  __syncthreads();
  const int n = k1 - k0;
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k0 + i, a.G, a.st, 0, a.Y);
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  for (int s = 0; s < n; ++s) {
    const int k = k0 + s;
    const int slot = s % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    const cplx<R>* Ck = Gk + pipe.gstride;
    const cplx<R>* Fk = Ck + 3 * wp;
    if (tid < W) {                       // v_k = f_k - C_k y_{k-1}
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r >= nr) break;
        cplx<R> v = Fk[r * wp + tid];
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int ee = tid + dx;
          if (ee >= 0 && ee < W) {
            const cplx<R> c = Ck[(dx + 1) * wp + tid];
            const cplx<R> y = ybuf[r * wp + ee];
            v.re -= c.re * y.re - c.im * y.im;
            v.im -= c.re * y.im + c.im * y.re;
          }
        }
        vbuf[r * wp + tid] = v;
      }
    }
    __syncthreads();
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_rows<R, NR>(Gk, W, vbuf, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          ybuf[r * wp + row] = acc[r];
          if (mode == 1) a.Y[((size_t)k * nr + r) * wp + row] = acc[r];
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k + pipe.stages, a.G, a.st, 0, a.Y);
  }
  if (mode == 0) {
    for (int i = tid; i < nr * wp; i += nthr) a.carry_f[(size_t)p * nr * wp + i] = ybuf[i];
    return;
  }
  if (!bwd1) return;
  // Backward recurrence from a zero start: x_k = y_k - G_k (B_k x_{k+1}).
  // The y rows were written above by this CTA (generic stores); they are read
  // with ordinary loads, one step ahead, never through TMA.  The pipeline
  // still brings G_k and B_k (its vector part, Y row k, is not used here).
  for (int i = tid; i < NR * wp; i += nthr) ybuf[i] = zero;   // x_{k1}
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k1 - 1 - i, a.G, a.st, 6, a.Y);
  cplx<R> ynext[NR];
  {
    const int row0 = grp;   // rows handled by this group in the first pass over rb
#pragma unroll
    for (int r = 0; r < NR; ++r)
      ynext[r] = (lane == 0 && row0 < W && r < nr) ? a.Y[((size_t)(k1 - 1) * nr + r) * wp + row0] : zero;
  }
  for (int s = 0; s < n; ++s) {
    const int k = k1 - 1 - s;
    const int slot = s % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    const cplx<R>* Bk = Gk + pipe.gstride;
    if (tid < W) {                       // w = B_k x_{k+1}
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r >= nr) break;
        cplx<R> v = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int ee = tid + dx;
          if (ee >= 0 && ee < W) cfma(v, Bk[(dx + 1) * wp + tid], ybuf[r * wp + ee]);
        }
        vbuf[r * wp + tid] = v;
      }
    }
    __syncthreads();
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      cplx<R> ycur[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) ycur[r] = ynext[r];
      if (rb + ngroups >= W) {           // last pass over rows: prefetch row k-1
        const int rowp = grp;
#pragma unroll
        for (int r = 0; r < NR; ++r)
          ynext[r] = (lane == 0 && rowp < W && r < nr && k > k0)
                         ? a.Y[((size_t)(k - 1) * nr + r) * wp + rowp] : zero;
      }
      if (rb > 0) {                      // rows beyond the first pass: plain load now
#pragma unroll
        for (int r = 0; r < NR; ++r)
          ycur[r] = (lane == 0 && row < W && r < nr) ? a.Y[((size_t)k * nr + r) * wp + row] : zero;
      }
      gemv_rows<R, NR>(Gk, W, vbuf, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          ybuf[r * wp + row] = ycur[r] - acc[r];
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k - pipe.stages, a.G, a.st, 6, a.Y);
  }
  for (int i = tid; i < nr * wp; i += nthr) a.carry_b[(size_t)p * nr * wp + i] = ybuf[i];
}

// Final backward recurrence over one segment from x_{k1} = carry_b[p+1]
// (last segment: zero), with the epilogue of Table 2.
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_bwd_kernel(SolveArgs<R> a) {
  const int p = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, ny = a.ny, nr = a.nr;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  const int k0 = a.seg[p], k1 = a.seg[p + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  Pipe<R> pipe;
  cplx<R>* vbuf;
  cplx<R>* xbuf;
  init_pipe<R>(pipe, smem_raw, a, NR, &vbuf, &xbuf);
  const cplx<R> zero = mk<R>(0, 0);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
  }
  for (int i = tid; i < NR * wp; i += nthr) {
    const int r = i / wp, e = i - r * wp;
    xbuf[i] = (p + 1 < a.P && r < nr) ? a.carry_b[((size_t)(p + 1) * nr + r) * wp + e] : zero;
  }
  __syncthreads();
  const int n = k1 - k0;
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k1 - 1 - i, a.G, a.st, 6, a.Y);
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  const Out<R>& o = a.out;
  for (int s = 0; s < n; ++s) {
    const int k = k1 - 1 - s;
    const int slot = s % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    const cplx<R>* Bk = Gk + pipe.gstride;
    const cplx<R>* Yk = Bk + 3 * wp;
    if (tid < W) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r >= nr) break;
        cplx<R> v = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int ee = tid + dx;
          if (ee >= 0 && ee < W) cfma(v, Bk[(dx + 1) * wp + tid], xbuf[r * wp + ee]);
        }
        vbuf[r * wp + tid] = v;
      }
    }
    __syncthreads();
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_rows<R, NR>(Gk, W, vbuf, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
        const int g = row - o.wl + o.lo;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          const cplx<R> x = Yk[r * wp + row] - acc[r];
          xbuf[r * wp + row] = x;
          if (o.raw) o.raw[((size_t)r * ny + k) * W + row] = x;
          if (o.u && g > o.ua && g <= o.ub) o.u[((size_t)r * ny + k) * o.nx + g] = x;
          if (o.B2 && (row == o.e2 || row == o.e2 + 1))
            o.B2[((size_t)(row - o.e2) * nr + r) * ny + k] = x;
          if (o.B4 && (row == o.e4 || row == o.e4 + 1))
            o.B4[((size_t)(row - o.e4) * nr + r) * ny + k] = x;
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k - pipe.stages, a.G, a.st, 6, a.Y);
  }
}

// Segment carries: forward Y_p = yhat_p + Phi_p Y_{p-1} (p = 1..P-1);
// backward X_p = xhat_p + Psi_p X_{p+1} (p = P-2..0).  The products and the
// segment values come through a TMA pipeline: stage = [M_p | carry row p].
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_carry_kernel(SolveArgs<R> a, const cplx<R>* prod,
                                                              int backward) {
  const int tid = threadIdx.x, W = a.W, wp = a.wp, nr = a.nr, P = a.P;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  uint64_t* bar = (uint64_t*)smem_raw;
  cplx<R>* prev = (cplx<R>*)(smem_raw + 128);
  cplx<R>* buf = (cplx<R>*)(((uintptr_t)(prev + NR * wp) + 127) & ~(uintptr_t)127);
  const size_t se = a.gstride + (size_t)nr * wp;
  const int stages = a.stages;
  cplx<R>* carry = backward ? a.carry_b : a.carry_f;
  const uint32_t mb = (uint32_t)(a.gstride * sizeof(cplx<R>));
  const uint32_t vb = (uint32_t)((size_t)nr * wp * sizeof(cplx<R>));
  auto seg_of = [&](int q) { return backward ? P - 1 - q : q; };
  auto issue = [&](int i, int q) {
    const int p = seg_of(q);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[i], mb + vb);
    tma_load_1d(buf + (size_t)i * se, prod + (size_t)p * a.gstride, mb, &bar[i]);
    tma_load_1d(buf + (size_t)i * se + a.gstride, carry + (size_t)p * nr * wp, vb, &bar[i]);
  };
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < stages; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  const int pstart = seg_of(0);
  for (int i = tid; i < NR * wp; i += nthr)
    prev[i] = (i < nr * wp) ? carry[(size_t)pstart * nr * wp + i] : mk<R>(0, 0);
  __syncthreads();
  const int n = P - 1;
  if (tid == 0)
    for (int i = 0; i < stages && i < n; ++i) issue(i, i + 1);
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  for (int s = 0; s < n; ++s) {
    const int q = s + 1;
    const int p = seg_of(q);
    const int slot = s % stages;
    if (!mbar_wait(&bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    __syncthreads();
    if (sh_abort) return;
    const cplx<R>* M = buf + (size_t)slot * se;
    const cplx<R>* hat = M + a.gstride;
    cplx<R> res[NR];
    int myrow = -1;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_rows<R, NR>(M, W, prev, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
        myrow = row;
#pragma unroll
        for (int r = 0; r < NR; ++r) res[r] = (r < nr) ? hat[r * wp + row] + acc[r] : mk<R>(0, 0);
      }
    }
    __syncthreads();   // everyone has read prev
    if (myrow >= 0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r >= nr) break;
        prev[r * wp + myrow] = res[r];
        carry[((size_t)p * nr + r) * wp + myrow] = res[r];
      }
    }
    __syncthreads();
    if (tid == 0 && s + stages < n) issue(slot, q + stages);
  }
}

// ------------------------------------------------------------------ host side
template <typename R>
static size_t solve_smem(const Slab& S, int nr, int NR, int stages) {
  const size_t el = sizeof(cplx<R>);
  size_t fixed = 128 + 2 * (size_t)NR * S.wp * el + 128;
  size_t stage = (S.gstride + 3 * (size_t)S.wp + (size_t)nr * S.wp) * el;
  return fixed + (size_t)stages * stage;
}

template <typename R>
static size_t carry_smem(const Slab& S, int nr, int NR, int stages) {
  const size_t el = sizeof(cplx<R>);
  return 128 + (size_t)NR * S.wp * el + 128 + (size_t)stages * (S.gstride + (size_t)nr * S.wp) * el;
}

constexpr size_t kSmemLimit = 225 * 1024;

template <typename R>
static int pick_stages(const Slab& S, int nr, int NR) {
  int st = 4;
  while (st > 1 && solve_smem<R>(S, nr, NR, st) > kSmemLimit) --st;
  if (solve_smem<R>(S, nr, NR, st) > kSmemLimit)
    throw Failure(HZ_EINVAL, "slab too wide for the shared-memory slab solve (W=" +
                                 std::to_string(S.W) + ")");
  return st;
}

template <typename R>
static int pick_carry_stages(const Slab& S, int nr, int NR) {
  int st = 4;
  while (st > 1 && carry_smem<R>(S, nr, NR, st) > kSmemLimit) --st;
  return st;
}

template <typename R>
void factor_level(hz_handle* h, Level& L, cudaStream_t s) {
  const int J = L.J;
  int maxW = 0;
  for (int j = 1; j <= J; ++j) maxW = std::max(maxW, L.slabs[j].W);
  size_t smem = 2 * (size_t)maxW * maxW * sizeof(cplx<R>) +
                (2 * FactorPanel<R>::BW + 9) * maxW * sizeof(cplx<R>) +
                FactorPanel<R>::BW * (sizeof(cplx<R>) + sizeof(int)) + 3 * maxW * sizeof(int) + 64;
  // register tiles of the delayed update: 4 x 4 while ceil(W/4)^2 <= block, else 4 x 8
  const int TC = ((maxW + 3) / 4) * ((maxW + 3) / 4) <= kThreads ? 4 : 8;
  if (((maxW + 3) / 4) * ((maxW + TC - 1) / TC) > kThreads || maxW > 128)
    throw Failure(HZ_EINVAL, "slab too wide for the blocked factorisation (W=" +
                                 std::to_string(maxW) + ")");
  std::vector<FactorDesc> fd(J);
  for (int j = 1; j <= J; ++j) {
    const Slab& S = L.slabs[j];
    fd[j - 1] = FactorDesc{S.W, S.wp, L.ny, S.st, S.G, S.gstride};
  }
  FactorDesc* d_fd = (FactorDesc*)dmalloc(sizeof(FactorDesc) * J);
  HZ_CU(cudaMemcpyAsync(d_fd, fd.data(), sizeof(FactorDesc) * J, cudaMemcpyHostToDevice, s));
  auto launch = [&](auto kern) {
    HZ_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timed(h, "slab_factor", 0.0, s, [&] { kern<<<J, kThreads, smem, s>>>(d_fd); });
  };
  if (TC == 4) launch(slab_factor_kernel<R, 4>);
  else launch(slab_factor_kernel<R, 8>);
  h->launches++;
  HZ_CU(cudaGetLastError());
  ProdDesc* d_pd = nullptr;
  if (L.P > 1) {
    std::vector<ProdDesc> pd;
    for (int j = 1; j <= J; ++j) {
      const Slab& S = L.slabs[j];
      for (int p = 0; p < L.P; ++p)
        for (int bw = 0; bw < 2; ++bw)
          pd.push_back(ProdDesc{S.W, S.wp, L.seg[p], L.seg[p + 1], bw, S.st, S.G, S.gstride,
                                (cplx<R>*)(bw ? S.Psi : S.Phi) + (size_t)p * S.gstride});
    }
    d_pd = (ProdDesc*)dmalloc(sizeof(ProdDesc) * pd.size());
    HZ_CU(cudaMemcpyAsync(d_pd, pd.data(), sizeof(ProdDesc) * pd.size(), cudaMemcpyHostToDevice, s));
    size_t psm = 2 * (size_t)maxW * maxW * sizeof(cplx<R>);
    HZ_CU(cudaFuncSetAttribute(segment_product_kernel<R>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    timed(h, "segment_product", 0.0, s, [&] {
      segment_product_kernel<R><<<(unsigned)pd.size(), kThreads, psm, s>>>(d_pd);
    });
    h->launches++;
    HZ_CU(cudaGetLastError());
  }
  HZ_CU(cudaStreamSynchronize(s));
  dfree(d_fd);
  dfree(d_pd);
}

template <typename R, int NR>
static void set_solve_attrs() {
  static bool done = false;
  if (done) return;
  HZ_CU(cudaFuncSetAttribute(slab_fwd_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  HZ_CU(cudaFuncSetAttribute(slab_bwd_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  HZ_CU(cudaFuncSetAttribute(slab_carry_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  done = true;
}

// Launch sequence of one slab solve; `tagged` brackets the kernels with
// timing events (when timing is on).
template <typename R, int NR>
static void launch_solve(hz_handle* h, Level& L, Slab& S, SolveArgs<R> a, cudaStream_t s,
                         bool tagged) {
  set_solve_attrs<R, NR>();
  const int P = L.P, nr = a.nr;
  a.stages = pick_stages<R>(S, nr, NR);
  const size_t smem = solve_smem<R>(S, nr, NR, a.stages);
  const double el = sizeof(cplx<R>);
  const double gbytes = (double)L.ny * S.W * S.W * el;          // one pass over G_0..G_{ny-1}
  const double cbytes = (double)L.ny * 3 * S.W * el;            // one pass over the couplings
  const double vbytes = (double)nr * L.ny * S.W * el;           // one slab-sized vector
  const double pbytes = (double)P * S.W * S.W * el;             // one set of segment products
  auto T = [&](const char* tag, double bytes, auto&& fn) {
    if (tagged) timed(h, tag, bytes, s, fn); else fn();
  };
  dim3 grid(P);
  // one 4-thread group per row of G: round W * kTPR up to whole warps
  const int nthr = std::min(kThreads, std::max(128, (S.W * kTPR + 31) / 32 * 32));
  const size_t gtotal = (size_t)L.ny * nr * S.wp;
  T("slab_gather", 2 * vbytes, [&] {
    slab_gather_kernel<R><<<cdiv(gtotal, 256), 256, 0, s>>>(a);
  });
  h->launches++;
  if (P == 1) {
    T("slab_fwd", gbytes + cbytes + 3 * vbytes, [&] {
      slab_fwd_kernel<R, NR><<<grid, nthr, smem, s>>>(a, 1, 0);
    });
    T("slab_bwd", gbytes + cbytes + 2 * vbytes, [&] {
      slab_bwd_kernel<R, NR><<<grid, nthr, smem, s>>>(a);
    });
    h->launches += 2;
  } else {
    SolveArgs<R> ac = a;
    ac.stages = pick_carry_stages<R>(S, nr, NR);
    const size_t csm = carry_smem<R>(S, nr, NR, ac.stages);
    T("slab_fwd_pass1", gbytes + cbytes + 3 * vbytes, [&] {
      slab_fwd_kernel<R, NR><<<grid, nthr, smem, s>>>(a, 0, 0);
    });
    T("slab_carry", pbytes, [&] {
      slab_carry_kernel<R, NR><<<1, nthr, csm, s>>>(ac, (const cplx<R>*)S.Phi, 0);
    });
    T("slab_fwd_bwd1", 2 * gbytes + 2 * cbytes + 4 * vbytes, [&] {
      slab_fwd_kernel<R, NR><<<grid, nthr, smem, s>>>(a, 1, 1);
    });
    T("slab_carry", pbytes, [&] {
      slab_carry_kernel<R, NR><<<1, nthr, csm, s>>>(ac, (const cplx<R>*)S.Psi, 1);
    });
    T("slab_bwd", gbytes + cbytes + 2 * vbytes, [&] {
      slab_bwd_kernel<R, NR><<<grid, nthr, smem, s>>>(a);
    });
    h->launches += 5;
  }
  HZ_CU(cudaGetLastError());
}

template <typename R>
static void run_solve(hz_handle* h, Level& L, Slab& S, const Rhs<R>& rhs, const Out<R>& out,
                      int n_rhs, cudaStream_t s, cplx<R>* Y, cplx<R>* cf, cplx<R>* cb,
                      bool tagged) {
  if (n_rhs < 1 || n_rhs > kNRMax) throw Failure(HZ_EINVAL, "right-hand sides per slab launch must be 1..8");
  SolveArgs<R> a;
  a.W = S.W; a.wp = S.wp; a.ny = L.ny; a.nr = n_rhs; a.P = L.P; a.seg = L.seg_dev;
  a.st = (const cplx<R>*)S.st; a.G = (const cplx<R>*)S.G; a.gstride = S.gstride;
  a.stages = 1;
  a.Y = Y; a.carry_f = cf; a.carry_b = cb;
  a.flag = h->dev_flag;
  a.rhs = rhs;
  a.out = out;
  const double el = sizeof(cplx<R>);
  auto seq = [&] {
    if (n_rhs == 1) launch_solve<R, 1>(h, L, S, a, s, tagged);
    else if (n_rhs == 2) launch_solve<R, 2>(h, L, S, a, s, tagged);
    else if (n_rhs <= 4) launch_solve<R, 4>(h, L, S, a, s, tagged);
    else launch_solve<R, 8>(h, L, S, a, s, tagged);
  };
  // whole subdomain solve; algorithmic bytes = the method's minimum: G and
  // the couplings read once per substitution direction, right-hand side and
  // solution once
  const double minimal = 2.0 * L.ny * S.W * (S.W + 3.0) * el + 2.0 * n_rhs * L.ny * S.W * el;
  if (tagged) timed(h, "slab_solve", minimal, s, seq); else seq();
}

template <typename R>
void subdom_solve(hz_handle* h, Level& L, int j, const cplx<R>* f, int a, int b, int at, int bt,
                  bool tau1, const cplx<R>* B1, bool tau2, cplx<R>* B2, bool tau3,
                  const cplx<R>* B3, bool tau4, cplx<R>* B4, cplx<R>* u, int n_rhs,
                  cudaStream_t s) {
  Slab& S = L.slabs[j];
  // transmission from or to a missing neighbour is dropped (T^(1) = T~^(J) = 0)
  tau1 = tau1 && j > 1;
  tau4 = tau4 && j > 1;
  tau2 = tau2 && j < L.J;
  tau3 = tau3 && j < L.J;
  auto loc = [&](int g) { return g - S.lo + S.wl; };
  Rhs<R> q{};
  q.raw = nullptr; q.f = f; q.nx = L.nx; q.lo = S.lo; q.wl = S.wl; q.ga = a; q.gb = b;
  q.B1 = B1; q.ef = tau1 ? loc(L.beta[j - 1]) : -1;
  q.B3 = B3; q.eb = tau3 ? loc(L.beta_t[j]) : -1;
  q.inj = (const cplx<R>*)S.inj;
  Out<R> o{};
  o.raw = nullptr; o.u = u; o.nx = L.nx; o.lo = S.lo; o.wl = S.wl; o.ua = at; o.ub = bt;
  o.B2 = tau2 ? B2 : nullptr; o.e2 = tau2 ? loc(L.beta[j]) : -1;
  o.B4 = tau4 ? B4 : nullptr; o.e4 = tau4 ? loc(L.beta_t[j - 1]) : -1;
  run_solve<R>(h, L, S, q, o, n_rhs, s, (cplx<R>*)S.Y, (cplx<R>*)S.carry_f, (cplx<R>*)S.carry_b,
               true);
}

template <typename R>
void slab_solve_raw(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud, int n_rhs,
                    cudaStream_t s) {
  Slab& S = L.slabs[j];
  Rhs<R> q{};
  q.raw = fd; q.ef = -1; q.eb = -1;
  Out<R> o{};
  o.raw = ud; o.e2 = -1; o.e4 = -1;
  run_solve<R>(h, L, S, q, o, n_rhs, s, (cplx<R>*)S.Y, (cplx<R>*)S.carry_f, (cplx<R>*)S.carry_b,
               true);
}

// Slab solve of a raw right-hand side with caller-provided work buffers
// (Y [ny][n_rhs][wp], segment carries [P][n_rhs][wp] each); the same kernels
// as slab_solve_raw, no allocation, no timing events.
template <typename R>
void slab_solve_raw_scratch(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud,
                            int n_rhs, cudaStream_t s, cplx<R>* Y, cplx<R>* carry_f,
                            cplx<R>* carry_b) {
  Slab& S = L.slabs[j];
  Rhs<R> q{};
  q.raw = fd; q.ef = -1; q.eb = -1;
  Out<R> o{};
  o.raw = ud; o.e2 = -1; o.e4 = -1;
  run_solve<R>(h, L, S, q, o, n_rhs, s, Y, carry_f, carry_b, false);
}

template void factor_level<float>(hz_handle*, Level&, cudaStream_t);
template void factor_level<double>(hz_handle*, Level&, cudaStream_t);
template void subdom_solve<float>(hz_handle*, Level&, int, const c64*, int, int, int, int, bool,
                                  const c64*, bool, c64*, bool, const c64*, bool, c64*, c64*, int,
                                  cudaStream_t);
template void subdom_solve<double>(hz_handle*, Level&, int, const c128*, int, int, int, int, bool,
                                   const c128*, bool, c128*, bool, const c128*, bool, c128*, c128*,
                                   int, cudaStream_t);
template void slab_solve_raw<float>(hz_handle*, Level&, int, const c64*, c64*, int, cudaStream_t);
template void slab_solve_raw<double>(hz_handle*, Level&, int, const c128*, c128*, int, cudaStream_t);
template void slab_solve_raw_scratch<float>(hz_handle*, Level&, int, const c64*, c64*, int,
                                            cudaStream_t, c64*, c64*, c64*);
template void slab_solve_raw_scratch<double>(hz_handle*, Level&, int, const c128*, c128*, int,
                                             cudaStream_t, c128*, c128*, c128*);

}  // namespace hz
