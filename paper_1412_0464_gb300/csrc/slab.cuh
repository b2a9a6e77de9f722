// Slab factorisation and slab solves (the subdomain solves of SubdomSolve,
// Table 2; the paper uses a sparse direct solver, Section 5).
//
// A^(j) is block tridiagonal along y with W x W blocks (one block row per
// grid row k): D_k couples row k to itself, C_k to row k-1, B_k to row k+1
// (taken from the slab stencil st[k][9][wp], plane (dy+1)*3 + (dx+1)).
//
// Twisted block LU.  Two elimination chains start at the two outer PML
// boundaries of the slab (rows 0 and ny-1) and meet at the row m = mid:
//   top     S_0 = D_0,         S_k = D_k - C_k G_{k-1} B_{k-1}   (k < m)
//   bottom  S_{ny-1} = D_{ny-1}, S_k = D_k - B_k G_{k+1} C_{k+1}   (k > m)
//   meeting S_m = D_m - C_m G_{m-1} B_{m-1} - B_m G_{m+1} C_{m+1},
// G_k = S_k^-1 (stored).  Every Schur complement of a chain belongs to a
// part of the slab that contains an absorbing layer, so no block inverse is
// that of a closed (possibly resonant) cavity, and the two chains run in
// parallel.
// Solve A^(j) x = f: along each chain (t = position, L_t / R_t the couplings
// to the previous / next row of the chain)
//   forward   y_t = G_t (f_t - L_t y_{t-1})
//   meeting   x_m = G_m (f_m - C_m y_{m-1} - B_m y_{m+1})
//   backward  x_t = y_t - G_t R_t x_{t+1}   (x after the last row: x_m).
// Parallel in y: each chain is cut into segments.  Both recurrences are
// affine, y_t = G_t f_t + F_t y_{t-1} (F_t = -G_t L_t) and
// x_t = y_t + E_t x_{t+1} (E_t = -G_t R_t).  Per segment the products
// Phi = F_last ... F_first and Psi = E_first ... E_last are formed at factor
// time; a solve runs each segment from a zero start (all segments of both
// chains in parallel), carries the segment end values through Phi / Psi, and
// re-runs each segment from its true start.  The carries are two-level: the
// segments of a half form groups of about sqrt(P/2); the carry inside every
// group runs from a zero group start (all groups in parallel), one short
// chain per half carries the group boundary values through the in-group
// prefix products PhiP / PsiP (formed with the factorisation), and each
// segment's true start follows from its in-group value by one more product
// with PhiP / PsiP in the prologue of the re-run.
//
// Every substitution step reads its operands -- the factor block G_k, the
// coupling row and the right-hand-side row -- through one stage of a
// shared-memory pipeline filled by TMA bulk copies (cp.async.bulk +
// mbarrier); the step itself touches only shared memory and registers.
//
// Templates only: slab_c64.cu and slab_c128.cu instantiate the complex64 and
// complex128 paths in two translation units compiled side by side.
#pragma once
#include "hz_internal.h"
#include "ptx.cuh"

#include <algorithm>
#include <type_traits>
#include <cmath>

namespace hz {

constexpr int kThreads = 512;
constexpr int kTPR = 4;                 // threads cooperating on one row of a GEMV
constexpr int kNRMax = 8;               // right-hand sides per launch

// --------------------------------------------------------------- factorisation
// Each S is inverted by Gauss-Jordan elimination with partial pivoting;
// pivot rows are marked, not moved, and the permutations are applied when the
// inverse is written: G[p][piv[q]] = S[piv[p]][q].  With colmod = column p of
// S except colmod[r] = S[r][p] - 1, and rowmod = row r of S scaled by
// inv = 1/S[r][p] except rowmod[p] = inv + 1, one elimination step (pivot row
// included) is the rank-1 update S -= colmod rowmod^T.  The steps are blocked
// by panels of BW columns: one warp eliminates the panel's BW pivots on the
// panel columns only (shuffles, no block barrier), the pivot rows' other
// columns follow from the short recurrence
// rowmod_t = (S[r_t] - sum_{s<t} colmod_s[r_t] rowmod_s) inv_t, and all
// threads apply the delayed rank-BW update S -= Cm^T R in row strips.
__device__ __forceinline__ cplx<float> crcp(cplx<float> a) {
  const float d = __frcp_rn(a.re * a.re + a.im * a.im);
  return mk(a.re * d, -a.im * d);
}
__device__ __forceinline__ cplx<double> crcp(cplx<double> a) {
  const double d = __drcp_rn(a.re * a.re + a.im * a.im);
  return mk(a.re * d, -a.im * d);
}

// Panel width of the Gauss-Jordan elimination: 4 pivots per panel (wider
// fully unrolled panels cost more per pivot on sm_103a, measured).
template <typename R>
struct FactorPanel { static constexpr int BW = 4; };

// Warps of the delayed Gauss-Jordan updates.  The 12 warps that do not share
// a scheduler with the panel warp 0 (warp w runs on sub-partition w mod 4)
// take strips of RPW consecutive rows; the three that do (warps 4, 8, 12)
// take at most one leftover row each, so that they take few issue slots from
// the latency-bound panel elimination beside them.
constexpr int kMainUpdateWarps = kThreads / 32 / 4 * 3;
constexpr int kLateUpdateWarps = kThreads / 32 / 4 - 1;
struct Strip {
  int row0;        // first row of this warp's strip, -1: no rows
  int nrows;       // rows of the strip (<= RPW)
  bool late;       // shares warp 0's sub-partition (at most one row)
};
template <int RPW>
__device__ __forceinline__ Strip strip_of(int tid, int W) {
  const int warp = tid >> 5;
  Strip s;
  s.late = warp != 0 && (warp & 3) == 0;
  if (warp == 0) {
    s.row0 = -1;
    s.nrows = 0;
  } else if (!s.late) {
    s.row0 = ((warp >> 2) * 3 + (warp & 3) - 1) * RPW;
    s.nrows = min(RPW, W - s.row0);
  } else {
    const int rest = max(0, W - kMainUpdateWarps * RPW);
    const int rps = (rest + kLateUpdateWarps - 1) / kLateUpdateWarps;
    s.row0 = kMainUpdateWarps * RPW + ((warp >> 2) - 1) * rps;
    s.nrows = min(rps, W - s.row0);
  }
  if (s.nrows <= 0) {
    s.row0 = -1;
    s.nrows = 0;
  }
  return s;
}


// dst = -A B (NEG) or A B for W x W operands (A with row stride lda in shared
// or global memory, read through L2 only if CG; B and dst dense W x W in
// shared memory), all kThreads
// threads: warp w takes rows w*RPW .. w*RPW+RPW-1, lane l takes columns l,
// l+32, ... (CPL of them).  A reads are broadcasts and B / dst accesses are
// consecutive across the warp, so no shared-memory access conflicts.  The
// caller synchronises.
template <typename R, int RPW, int CPL, bool NEG = true, bool CG = false>
__device__ __forceinline__ void gemm_strip(const cplx<R>* A, int lda, const cplx<R>* B,
                                           cplx<R>* dst, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = warp * RPW;
  if (i0 >= W) return;
  const cplx<R> zero = mk<R>(0, 0);
  cplx<R> acc[RPW][CPL];
#pragma unroll
  for (int a = 0; a < RPW; ++a)
#pragma unroll
    for (int b = 0; b < CPL; ++b) acc[a][b] = zero;
  for (int l = 0; l < W; ++l) {
    cplx<R> bv[CPL];
#pragma unroll
    for (int b = 0; b < CPL; ++b) {
      const int j = lane + 32 * b;
      bv[b] = (j < W) ? B[l * W + j] : zero;
    }
#pragma unroll
    for (int a = 0; a < RPW; ++a) {
      const cplx<R> av = (i0 + a < W) ? (CG ? ldcg(A + (i0 + a) * lda + l) : A[(i0 + a) * lda + l])
                                      : zero;
#pragma unroll
      for (int b = 0; b < CPL; ++b) cfma(acc[a][b], av, bv[b]);
    }
  }
#pragma unroll
  for (int a = 0; a < RPW; ++a)
#pragma unroll
    for (int b = 0; b < CPL; ++b) {
      const int i = i0 + a, j = lane + 32 * b;
      if (i < W && j < W) dst[i * W + j] = NEG ? -acc[a][b] : acc[a][b];
    }
}

// One warp eliminates pivots p0 .. p0+bw-1 on the panel columns p0 .. p0+bw-1
// (rows lane + 32 m, m < MR, in registers) and records colmod (Cm), the pivot
// inverses and rows.  The panel columns first receive the pending rank-pbw
// update of the previous panel, S -= Cp^T Rp (pbw = 0: none).
template <typename R, int BW, int MR>
__device__ __forceinline__ void panel_elim(cplx<R>* S, cplx<R>* Cm, const cplx<R>* Cp,
                                           const cplx<R>* Rp, int pbw, cplx<R>* pinv, int* prow,
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
  for (int t = 0; t < pbw; ++t) {
    cplx<R> cv[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) cv[m] = (lane + 32 * m < W) ? Cp[t * W + lane + 32 * m] : zero;
#pragma unroll
    for (int c = 0; c < BW; ++c) {
      const cplx<R> rv = (c < bw) ? Rp[t * W + p0 + c] : zero;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        P[m][c].re -= cv[m].re * rv.re - cv[m].im * rv.im;
        P[m][c].im -= cv[m].re * rv.im + cv[m].im * rv.re;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < BW; ++t) {
    if (t < bw) {
      // pivot row: largest |S[i][p]|^2 over the unused rows, by one max
      // reduction over keys = float bits of |S|^2 (low 8 bits dropped, a
      // 2^-15 relative tie width) | 0x80 | row.  Every unused row offers a key
      // > 0 (NaN or zero entries included), so a valid row always wins.
      unsigned key = 0u;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        if (!usd[m]) {
          const float v = (float)cabs2(P[m][t]);
          const unsigned row = (unsigned)(lane + 32 * m) | 0x80u;
          const unsigned kv = (v > 0.0f) ? ((__float_as_uint(v) & ~255u) | row) : row;
          key = max(key, kv);
        }
      }
      const int r = (int)(__reduce_max_sync(0xffffffffu, key) & 127u);
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

template <typename R, int BW>
__device__ __forceinline__ void panel_dispatch(cplx<R>* S, cplx<R>* Cm, const cplx<R>* Cp,
                                               const cplx<R>* Rp, int pbw, cplx<R>* pinv,
                                               int* prow, int* piv, int* used, int W, int p0,
                                               int bw, int lane) {
  const int MR = (W + 31) >> 5;
  if (MR == 1)
    panel_elim<R, BW, 1>(S, Cm, Cp, Rp, pbw, pinv, prow, piv, used, W, p0, bw, lane);
  else if (MR == 2)
    panel_elim<R, BW, 2>(S, Cm, Cp, Rp, pbw, pinv, prow, piv, used, W, p0, bw, lane);
  else if (MR == 3)
    panel_elim<R, BW, 3>(S, Cm, Cp, Rp, pbw, pinv, prow, piv, used, W, p0, bw, lane);
  else
    panel_elim<R, BW, 4>(S, Cm, Cp, Rp, pbw, pinv, prow, piv, used, W, p0, bw, lane);
}

// Delayed rank-pbw update S -= Cp^T Rm on rows row0 .. row0+nrows-1 (nrows <=
// RPW) and columns lane + 32 b outside panels q-1 (from pp0) and q (p0, bw):
// one warp.  The pbw x CPL rowmod values of this lane's columns stay in
// registers; the rows are updated one after the other (CPL accumulators),
// with the colmod entries of a row read as broadcasts.
template <typename R, int CPL, int BW>
__device__ __forceinline__ void strip_row(cplx<R>* Srow, const cplx<R>* Cp, int W, int i,
                                          const cplx<R> (&rv)[BW][CPL], const bool (&ok)[CPL],
                                          int pbw) {
  cplx<R> x[CPL];
#pragma unroll
  for (int b = 0; b < CPL; ++b) x[b] = ok[b] ? Srow[32 * b] : mk<R>(0, 0);
#pragma unroll
  for (int t = 0; t < BW; ++t) {
    const cplx<R> cv = (t < pbw) ? Cp[t * W + i] : mk<R>(0, 0);   // same address across the warp
#pragma unroll
    for (int b = 0; b < CPL; ++b) {
      x[b].re -= cv.re * rv[t][b].re - cv.im * rv[t][b].im;
      x[b].im -= cv.re * rv[t][b].im + cv.im * rv[t][b].re;
    }
  }
#pragma unroll
  for (int b = 0; b < CPL; ++b)
    if (ok[b]) Srow[32 * b] = x[b];
}

template <typename R, int RPW, int CPL, int BW>
__device__ __forceinline__ void strip_update(cplx<R>* S, const cplx<R>* Cp, const cplx<R>* Rm,
                                             int W, int row0, int nrows, int pp0, int p0, int bw,
                                             int pbw, int lane) {
  bool ok[CPL];
#pragma unroll
  for (int b = 0; b < CPL; ++b) {
    const int j = lane + 32 * b;
    ok[b] = j < W && (j < pp0 || j >= p0 + bw);
  }
  cplx<R> rv[BW][CPL];
#pragma unroll
  for (int t = 0; t < BW; ++t)
#pragma unroll
    for (int b = 0; b < CPL; ++b)
      rv[t][b] = (t < pbw && ok[b]) ? Rm[t * W + lane + 32 * b] : mk<R>(0, 0);
  cplx<R>* S0 = S + (size_t)row0 * W + lane;
  if (nrows == RPW) {
#pragma unroll
    for (int a = 0; a < RPW; ++a) strip_row<R, CPL, BW>(S0 + a * W, Cp, W, row0 + a, rv, ok, pbw);
  } else {
    for (int a = 0; a < nrows; ++a) strip_row<R, CPL, BW>(S0 + a * W, Cp, W, row0 + a, rv, ok, pbw);
  }
}

// Shared-memory work areas of the Gauss-Jordan inverse.
template <typename R>
struct GJWork {
  cplx<R>* Cm;     // 2 x BW x W (colmods of two consecutive panels)
  cplx<R>* Rm;     // BW x W
  cplx<R>* pinv;   // BW
  int* prow;       // BW
  int* piv;        // W
  int* ipiv;       // W
  int* used;       // W
};

// S^-1 (S: W x W in shared memory, overwritten) into `out` (global) and Gl
// (shared), both in natural order.  Called by every thread of a kThreads
// block after a barrier that completes S; ends with a barrier.  `su` is this
// warp's row strip in the delayed updates (update warps only; lane l holds
// columns l, l + 32, ..., so every shared-memory access of the update is
// conflict-free or a broadcast).
//
// Look-ahead: while warp 0 applies panel q-1's pending update to the columns
// of panel q and eliminates panel q, the update warps apply the same update to
// all other columns; then all threads form the pivot rows of panel q (rowmod).
// Two block barriers per panel.
template <typename R, int RPW, int CPL>
__device__ void gj_inverse(cplx<R>* S, cplx<R>* Gl, const GJWork<R>& w, int W, const Strip& su,
                           cplx<R>* out) {
  constexpr int BW = FactorPanel<R>::BW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int WW = W * W;
  const int NP = (W + BW - 1) / BW;
  const cplx<R> zero = mk<R>(0, 0);
  for (int t = tid; t < W; t += kThreads) w.used[t] = 0;
  __syncthreads();
  for (int q = 0; q <= NP; ++q) {
    const int p0 = q * BW, bw = (q < NP) ? min(BW, W - p0) : 0;       // panel q (to eliminate)
    const int pp0 = (q - 1) * BW, pbw = (q > 0) ? min(BW, W - pp0) : 0;   // panel q-1 (pending)
    cplx<R>* Cq = w.Cm + (size_t)(q & 1) * BW * W;
    const cplx<R>* Cp = w.Cm + (size_t)((q + 1) & 1) * BW * W;
    if (warp == 0) {
      if (bw > 0)
        panel_dispatch<R, BW>(S, Cq, Cp, w.Rm, pbw, w.pinv, w.prow, w.piv, w.used, W, p0, bw, lane);
    } else if (pbw > 0 && su.row0 >= 0) {
      // delayed rank-pbw update of panel q-1 on every column outside panels
      // q-1 and q (a late warp has at most one row: a one-row tile)
      if (su.late)
        strip_update<R, 1, CPL, BW>(S, Cp, w.Rm, W, su.row0, su.nrows, pp0, p0, bw, pbw, lane);
      else
        strip_update<R, RPW, CPL, BW>(S, Cp, w.Rm, W, su.row0, su.nrows, pp0, p0, bw, pbw, lane);
    }
    __syncthreads();
    if (bw == 0) break;
    // rowmod of panel q's pivots on the other columns (one thread per column,
    // W <= kThreads): R_t = (S[r_t] - sum_{s<t} colmod_s[r_t] R_s) inv_t.  All
    // operands are loaded before the short recurrence runs.
    if (tid < W && (tid < p0 || tid >= p0 + bw)) {
      const int j = tid;
      int r[BW];
      cplx<R> u[BW], iv[BW], c[BW][BW];
#pragma unroll
      for (int t = 0; t < BW; ++t) r[t] = (t < bw) ? w.prow[t] : 0;
#pragma unroll
      for (int t = 0; t < BW; ++t) {
        u[t] = S[r[t] * W + j];
        iv[t] = w.pinv[t];
#pragma unroll
        for (int s2 = 0; s2 < t; ++s2) c[t][s2] = Cq[s2 * W + r[t]];
      }
      cplx<R> rw[BW];
#pragma unroll
      for (int t = 0; t < BW; ++t) {
        if (t >= bw) break;
        cplx<R> acc = u[t];
#pragma unroll
        for (int s2 = 0; s2 < t; ++s2) {
          acc.re -= c[t][s2].re * rw[s2].re - c[t][s2].im * rw[s2].im;
          acc.im -= c[t][s2].re * rw[s2].im + c[t][s2].im * rw[s2].re;
        }
        rw[t] = acc * iv[t];
        w.Rm[t * W + j] = rw[t];
      }
    }
    __syncthreads();
  }
  for (int q = tid; q < W; q += kThreads) w.ipiv[w.piv[q]] = q;
  __syncthreads();
  for (int e = tid; e < WW; e += kThreads) {
    const int i = e / W, j = e - i * W;
    const cplx<R> v = S[w.piv[i] * W + w.ipiv[j]];
    out[e] = v;
    Gl[e] = v;
  }
  __syncthreads();
}

// Shared-memory layout of the factor kernels: S, Gl (W x W each), the
// Gauss-Jordan work, then `ncpl` coupling rows of W.
template <typename R>
__device__ __forceinline__ void factor_smem(unsigned char* raw, int W, int ncpl, cplx<R>** S,
                                            cplx<R>** Gl, GJWork<R>* w, cplx<R>** cpl) {
  constexpr int BW = FactorPanel<R>::BW;
  cplx<R>* p = (cplx<R>*)raw;
  *S = p;
  *Gl = p + W * W;
  w->Cm = *Gl + W * W;
  w->Rm = w->Cm + 2 * BW * W;
  *cpl = w->Rm + BW * W;
  w->pinv = *cpl + ncpl * W;
  w->prow = (int*)(w->pinv + BW);
  w->piv = w->prow + BW;
  w->ipiv = w->piv + W;
  w->used = w->ipiv + W;
}
static size_t factor_smem_bytes(int W, int ncpl, size_t el, int BW) {
  return (2 * (size_t)W * W + (3 * (size_t)BW + ncpl) * W + BW) * el + (BW + 3 * (size_t)W) * 4 + 64;
}

// Interior chains of the twisted factorisation (one CTA per slab and half).
// The chain visits rows k_t = k0 + dir t, t = 0..n-1, starting at the outer
// PML row (top half: k0 = 0, dir = +1; bottom half: k0 = ny-1, dir = -1):
//   S_0 = D_{k_0},  S_t = D_{k_t} - L_t G_{t-1} R_{t-1},  G_t = S_t^-1,
// with L_t the coupling of row k_t to the previous row of the chain (C_k for
// dir = +1, B_k for dir = -1) and R_{t-1} that of row k_{t-1} to k_t.
struct FactorDesc {
  int W, wp, k0, n, dir;
  int diag;                  // couplings L, R diagonal (5-point stencil): one-pass Schur update
  const void* st;
  void* G;
  size_t gstride;
};

__host__ __device__ __forceinline__ int lplane(int dir) { return dir > 0 ? 0 : 6; }
__host__ __device__ __forceinline__ int rplane(int dir) { return dir > 0 ? 6 : 0; }

// Asynchronous global -> shared copy of one complex element (cp.async); the
// copies of a thread complete at its cp_async_wait_all.
template <typename R>
__device__ __forceinline__ void cp_async_el(cplx<R>* dst, const cplx<R>* src) {
  if constexpr (sizeof(cplx<R>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Release store / acquire load of a progress counter (gpu scope).
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One elimination chain; if `progress` is given, the number of finished rows
// is published there (release) after every fourth G_t and the last one.
template <typename R, int RPW, int CPL>
__device__ void factor_chain(const FactorDesc& d, int* progress) {
  const int W = d.W, wp = d.wp, tid = threadIdx.x, dir = d.dir;
  const int WW = W * W;
  const Strip su = strip_of<RPW>(tid, W);
  const cplx<R>* st = (const cplx<R>*)d.st;
  cplx<R>* G = (cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>*S, *Gl, *cpl;
  GJWork<R> w;
  factor_smem<R>(smem_raw, W, 18, &S, &Gl, &w, &cpl);
  const cplx<R> zero = mk<R>(0, 0);
  const int pl = lplane(dir), pr = rplane(dir);
  cplx<R>* Gp = Gl;                              // G_{t-1}
  cplx<R>* Sp = S;                               // the other W x W buffer
  // couplings of row t in buffer t & 1: L_t, D_t, R_{t-1} (3 x W each); those
  // of row t+1 are copied (cp.async) while row t is inverted
  auto stage = [&](cplx<R>* cb, int t, bool async) {
    const int k = d.k0 + dir * t;
    const cplx<R>* stk = st + (size_t)k * 9 * wp;
    const cplx<R>* stp = st + (size_t)(k - dir) * 9 * wp;
    for (int i = tid; i < 3 * W; i += kThreads) {
      const int q = i / W, e = i - q * W;
      if (async) {
        cp_async_el(cb + i, stk + (pl + q) * wp + e);
        cp_async_el(cb + 3 * W + i, stk + (3 + q) * wp + e);
        cp_async_el(cb + 6 * W + i, stp + (pr + q) * wp + e);
      } else {
        cb[i] = stk[(pl + q) * wp + e];
        cb[3 * W + i] = stk[(3 + q) * wp + e];
        cb[6 * W + i] = (t > 0) ? stp[(pr + q) * wp + e] : zero;
      }
    }
    if (async) cp_async_commit();
  };
  stage(cpl, 0, false);

  for (int t = 0; t < d.n; ++t) {
    const int k = d.k0 + dir * t;
    cplx<R>* cL = cpl + (t & 1) * 9 * W;           // L_t (3 x W)
    cplx<R>* cD = cL + 3 * W;                      // D (3 x W)
    cplx<R>* cR = cD + 3 * W;                      // R_{t-1} (3 x W)
    if (t > 0) cp_async_wait_all();
    __syncthreads();
    // Gp holds G_{t-1}; S_t is formed in the other buffer (or, for
    // tridiagonal couplings, in Gp after X = G_{t-1} R_{t-1} went to the
    // other), inverted in place, and G_t lands in the remaining one.
    cplx<R>* Sx = Sp;        // S_t
    cplx<R>* Gx = Gp;        // receives G_t
    if (t > 0 && d.diag) {
      for (int e = tid; e < WW; e += kThreads) {      // S_t = D - L_t G_{t-1} R_{t-1}
        const int i = e / W, j = e - i * W;
        cplx<R> v = -(cL[W + i] * Gp[e] * cR[W + j]);
        const int dd = j - i;
        if (dd >= -1 && dd <= 1) v = v + cD[(dd + 1) * W + i];
        Sp[e] = v;
      }
    } else if (t > 0) {
      for (int e = tid; e < WW; e += kThreads) {      // X = G_{t-1} R_{t-1} into Sp
        const int i = e / W, j = e - i * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int c = j - dx;
          if (c >= 0 && c < W) cfma(acc, Gp[i * W + c], cR[(dx + 1) * W + c]);
        }
        Sp[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < WW; e += kThreads) {      // S_t = D - L X into Gp
        const int i = e / W, j = e - i * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int rr = i + dx;
          if (rr >= 0 && rr < W) cfma(acc, cL[(dx + 1) * W + i], Sp[rr * W + j]);
        }
        cplx<R> v = -acc;
        const int dd = j - i;
        if (dd >= -1 && dd <= 1) v = v + cD[(dd + 1) * W + i];
        Gp[e] = v;
      }
      Sx = Gp;
      Gx = Sp;
    } else {
      for (int e = tid; e < WW; e += kThreads) {
        const int i = e / W, j = e - i * W;
        const int dd = j - i;
        Sp[e] = (dd >= -1 && dd <= 1) ? cD[(dd + 1) * W + i] : zero;
      }
    }
    __syncthreads();
    if (t + 1 < d.n) stage(cpl + ((t + 1) & 1) * 9 * W, t + 1, true);
    gj_inverse<R, RPW, CPL>(Sx, Gx, w, W, su, G + (size_t)k * d.gstride);
    Gp = Gx;
    Sp = Sx;
    // every thread's G_t stores precede the barrier that ends gj_inverse; the
    // fence stalls thread 0 (and through the next barrier the chain), so the
    // progress is published every 4 rows and at the last row
    if (progress && tid == 0 && (((t + 1) & 3) == 0 || t + 1 == d.n)) {
      __threadfence();
      st_release(progress, t + 1);
    }
  }
}

template <typename R, int RPW, int CPL>
__global__ void __launch_bounds__(kThreads) slab_factor_kernel(const FactorDesc* descs) {
  factor_chain<R, RPW, CPL>(descs[blockIdx.x], nullptr);
}

// sum_{dx, dy} Lc[dx][i] X[i+dx][j-dy] Rc[dy][j-dy]: (L X R)[i][j] for
// tridiagonal L (row i: Lc[(dx+1) W + i] at column i+dx) and R.
template <typename R>
__device__ __forceinline__ cplx<R> tri_x_tri(const cplx<R>* Lc, const cplx<R>* X, const cplx<R>* Rc,
                                             int W, int i, int j) {
  cplx<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int dx = -1; dx <= 1; ++dx) {
    const int r = i + dx;
    if (r < 0 || r >= W) continue;
    cplx<R> xr = mk<R>(0, 0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int l = j - dy;
      if (l >= 0 && l < W) cfma(xr, X[r * W + l], Rc[(dy + 1) * W + l]);
    }
    cfma(acc, Lc[(dx + 1) * W + i], xr);
  }
  return acc;
}

// The meeting row m of the two chains (one CTA per slab):
//   S_m = D_m - C_m G_{m-1} B_{m-1} - B_m G_{m+1} C_{m+1},  G_m = S_m^-1.
struct MidDesc {
  int W, wp, m;
  const void* st;
  void* G;
  size_t gstride;
};

template <typename R, int RPW, int CPL>
__global__ void __launch_bounds__(kThreads) slab_middle_kernel(const MidDesc* descs) {
  const MidDesc d = descs[blockIdx.x];
  const int W = d.W, wp = d.wp, m = d.m, tid = threadIdx.x, WW = W * W;
  const Strip su = strip_of<RPW>(tid, W);
  const cplx<R>* st = (const cplx<R>*)d.st;
  cplx<R>* G = (cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>*S, *Gl, *cpl;
  GJWork<R> w;
  factor_smem<R>(smem_raw, W, 15, &S, &Gl, &w, &cpl);
  cplx<R>* Cm = cpl;            // C_m, D_m, B_m, B_{m-1}, C_{m+1}: 3 x W each
  cplx<R>* Dm = Cm + 3 * W;
  cplx<R>* Bm = Dm + 3 * W;
  cplx<R>* Bu = Bm + 3 * W;
  cplx<R>* Cd = Bu + 3 * W;
  for (int i = tid; i < 3 * W; i += kThreads) {
    const int q = i / W, e = i - q * W;
    const cplx<R>* sm = st + (size_t)m * 9 * wp;
    Cm[i] = sm[q * wp + e];
    Dm[i] = sm[(3 + q) * wp + e];
    Bm[i] = sm[(6 + q) * wp + e];
    Bu[i] = st[(size_t)(m - 1) * 9 * wp + (6 + q) * wp + e];
    Cd[i] = st[(size_t)(m + 1) * 9 * wp + q * wp + e];
  }
  __syncthreads();
  const cplx<R>* Gu = G + (size_t)(m - 1) * d.gstride;
  const cplx<R>* Gd = G + (size_t)(m + 1) * d.gstride;
  for (int e = tid; e < WW; e += kThreads) {
    const int i = e / W, j = e - i * W;
    const int dd = j - i;
    cplx<R> v = (dd >= -1 && dd <= 1) ? Dm[(dd + 1) * W + i] : mk<R>(0, 0);
    S[e] = v - tri_x_tri<R>(Cm, Gu, Bu, W, i, j) - tri_x_tri<R>(Bm, Gd, Cd, W, i, j);
  }
  __syncthreads();
  gj_inverse<R, RPW, CPL>(S, Gl, w, W, su, G + (size_t)m * d.gstride);
}

// Substitution operators and segment transfer products (one CTA per slab,
// segment and direction; all independent).  Along a segment's chain positions
// t = 0..n-1 the CTA forms and stores
//   forward  F'_t = G_t L_t   (y_t = g_t - F'_t y_{t-1})
//   backward E'_t = G_t R_t   (x_t = y_t - E'_t x_{t+1})
// (L_t / R_t: the tridiagonal coupling of row k_t to the previous / next row
// of its chain), and, if `chain`, the segment products
//   Phi = (-F'_{n-1}) ... (-F'_0),   Psi = (-E'_0) ... (-E'_{n-1}).
struct ProdDesc {
  int W, wp, k0, n, dir, backward, chain;
  int stage;                 // 1: A_t also kept in shared memory for the GEMM
  int fchain, need;          // elimination chain of the rows and rows it must have finished
  const void* st;
  const void* G;             // [ny][gstride], dense W x W
  void* A;                   // F' (forward) or E' (backward), [ny][mstride], row stride wp
  size_t gstride, mstride;
  void* out;                 // Phi or Psi block, row stride wp
  // fused launch only: a product task counts itself done in group counter
  // `gctr`; a prefix task (prefix = 1: the in-group prefix products of one
  // group and direction, k0 = first segment, n = segments, dir = +-1, from the
  // products in A to `out`) waits until counter `gctr` reaches `gneed`
  int prefix, gctr, gneed;
};

template <typename R, int RPW, int CPL>
__device__ void product_task(const ProdDesc& d) {
  const int W = d.W, wp = d.wp, tid = threadIdx.x, WW = W * W;
  const cplx<R>* st = (const cplx<R>*)d.st;
  const cplx<R>* G = (const cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* M = (cplx<R>*)smem_raw;
  cplx<R>* T = M + WW;
  cplx<R>* cp = T + WW;               // coupling (3 x W)
  cplx<R>* As = cp + 3 * W;           // A_t (if d.stage)
  const cplx<R> zero = mk<R>(0, 0);
  const int plane = d.backward ? rplane(d.dir) : lplane(d.dir);
  if (d.chain) {
    for (int e = tid; e < WW; e += kThreads) M[e] = (e / W == e % W) ? mk<R>(1, 0) : zero;
  }
  for (int s = 0; s < d.n; ++s) {
    const int t = d.backward ? d.n - 1 - s : s;
    const int k = d.k0 + d.dir * t;
    for (int i = tid; i < 3 * W; i += kThreads) {
      const int q = i / W, e = i - q * W;
      cp[i] = st[(size_t)k * 9 * wp + (plane + q) * wp + e];
    }
    __syncthreads();
    const cplx<R>* Gk = G + (size_t)k * d.gstride;
    cplx<R>* Ak = (cplx<R>*)d.A + (size_t)k * d.mstride;
    for (int e = tid; e < WW; e += kThreads) {        // A_t = G_t Cpl_t
      const int i = e / W, j = e - i * W;
      cplx<R> acc = zero;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int c = j - dx;
        if (c >= 0 && c < W) cfma(acc, ldcg(Gk + i * W + c), cp[(dx + 1) * W + c]);
      }
      if (d.stage) As[e] = acc;
      Ak[i * wp + j] = acc;
    }
    __syncthreads();
    if (d.chain) {                                   // T = -A_t M
      if (d.stage) gemm_strip<R, RPW, CPL>(As, W, M, T, W);
      else gemm_strip<R, RPW, CPL>(Ak, wp, M, T, W);
      __syncthreads();
      cplx<R>* x = M;
      M = T;
      T = x;
    }
  }
  if (d.chain) {
    cplx<R>* out = (cplx<R>*)d.out;
    for (int e = tid; e < WW; e += kThreads) out[(e / W) * wp + e % W] = M[e];
  }
}

template <typename R, int RPW, int CPL>
__global__ void __launch_bounds__(kThreads) segment_product_kernel(const ProdDesc* descs) {
  product_task<R, RPW, CPL>(descs[blockIdx.x]);
}

// In-group prefix products of the segment transfer products (one CTA per
// group and direction): along the group's segments in carry order
// q_0, q_1, ... (increasing q for Phi, decreasing for Psi)
//   Pi_{q_0} = M_{q_0},   Pi_{q_i} = M_{q_i} Pi_{q_{i-1}},
// so that a segment value of the carry recurrence v_q = vhat_q + M_q v_prev
// follows from its in-group value (zero start) as v_q = v_q^loc + Pi_q v_in,
// v_in the value entering the group.
struct PrefixDesc {
  int W, wp, q0, n, dir;
  const void* src;            // Phi or Psi [P][mstride]
  void* dst;                  // PhiP or PsiP [P][mstride]
  size_t mstride;
};

template <typename R, int RPW, int CPL>
__global__ void __launch_bounds__(kThreads) segment_prefix_kernel(const PrefixDesc* descs) {
  const PrefixDesc d = descs[blockIdx.x];
  const int W = d.W, wp = d.wp, tid = threadIdx.x, WW = W * W;
  const cplx<R>* src = (const cplx<R>*)d.src;
  cplx<R>* dst = (cplx<R>*)d.dst;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* M = (cplx<R>*)smem_raw;
  cplx<R>* T = M + WW;
  {
    const cplx<R>* s0 = src + (size_t)d.q0 * d.mstride;
    cplx<R>* d0 = dst + (size_t)d.q0 * d.mstride;
    for (int e = tid; e < WW; e += kThreads) {
      const int i = e / W, j = e - i * W;
      const cplx<R> v = ldcg(s0 + i * wp + j);
      M[e] = v;
      d0[i * wp + j] = v;
    }
  }
  __syncthreads();
  for (int i = 1; i < d.n; ++i) {
    const int q = d.q0 + d.dir * i;
    gemm_strip<R, RPW, CPL, false>(src + (size_t)q * d.mstride, wp, M, T, W);
    __syncthreads();
    cplx<R>* out = dst + (size_t)q * d.mstride;
    for (int e = tid; e < WW; e += kThreads) out[(e / W) * wp + e % W] = T[e];
    cplx<R>* x = M;
    M = T;
    T = x;
  }
}

// In-group prefix products of one group and direction (see
// segment_prefix_kernel) inside the fused launch: the products were written
// by other CTAs of the same launch, so they are read through L2 only.
template <typename R, int RPW, int CPL>
__device__ void prefix_task(const ProdDesc& d) {
  const int W = d.W, wp = d.wp, tid = threadIdx.x, WW = W * W;
  const cplx<R>* src = (const cplx<R>*)d.A;
  cplx<R>* dst = (cplx<R>*)d.out;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* M = (cplx<R>*)smem_raw;
  cplx<R>* T = M + WW;
  {
    const cplx<R>* s0 = src + (size_t)d.k0 * d.mstride;
    cplx<R>* d0 = dst + (size_t)d.k0 * d.mstride;
    for (int e = tid; e < WW; e += kThreads) {
      const int i = e / W, j = e - i * W;
      const cplx<R> v = ldcg(s0 + i * wp + j);
      M[e] = v;
      d0[i * wp + j] = v;
    }
  }
  __syncthreads();
  for (int i = 1; i < d.n; ++i) {
    const int q = d.k0 + d.dir * i;
    gemm_strip<R, RPW, CPL, false, true>(src + (size_t)q * d.mstride, wp, M, T, W);
    __syncthreads();
    cplx<R>* out = dst + (size_t)q * d.mstride;
    for (int e = tid; e < WW; e += kThreads) out[(e / W) * wp + e % W] = T[e];
    cplx<R>* x = M;
    M = T;
    T = x;
  }
}

// Factorisation and products in one cooperative launch (all CTAs resident):
// CTAs 0..nf-1 run the elimination chains and publish their progress; the
// others take product tasks in readiness order and wait (bounded by wait_ns,
// 10 s unless a test shortens it, then the device flag) until the chain has
// finished the task's rows.  A worker that gives up returns; the chains never
// wait, so the launch always ends.
template <typename R, int RPW, int CPL, int PRPW, int PCPL>
__global__ void __launch_bounds__(kThreads) slab_factor_fused_kernel(
    const FactorDesc* fd, int nf, const ProdDesc* pd, int np, int* progress, int* next_task,
    int* gdone, int* flag, unsigned long long wait_ns) {
  if ((int)blockIdx.x < nf) {
    factor_chain<R, RPW, CPL>(fd[blockIdx.x], progress + blockIdx.x);
    return;
  }
  __shared__ int sh_task, sh_abort;
  while (true) {
    if (threadIdx.x == 0) {
      sh_task = atomicAdd(next_task, 1);
      sh_abort = 0;
      if (sh_task < np) {
        const ProdDesc& d = pd[sh_task];
        if (ld_acquire(progress + d.fchain) < d.need) {
          const uint64_t t0 = gtimer();
          while (ld_acquire(progress + d.fchain) < d.need) {
            __nanosleep(2000);
            if (gtimer() - t0 > wait_ns) {
              atomicExch(flag, DEV_TIMEOUT);
              sh_abort = 1;
              break;
            }
          }
        }
        // a prefix task also waits for its group's products (all of them
        // precede it in the task order, so resident CTAs hold them)
        if (!sh_abort && d.prefix && ld_acquire(gdone + d.gctr) < d.gneed) {
          const uint64_t t0 = gtimer();
          while (ld_acquire(gdone + d.gctr) < d.gneed) {
            __nanosleep(1000);
            if (gtimer() - t0 > wait_ns) {
              atomicExch(flag, DEV_TIMEOUT);
              sh_abort = 1;
              break;
            }
          }
        }
      }
    }
    __syncthreads();
    const int task = sh_task;
    if (task >= np || sh_abort) return;
    const ProdDesc& d = pd[task];
    if (d.prefix) {
      prefix_task<R, PRPW, PCPL>(d);
    } else {
      product_task<R, PRPW, PCPL>(d);
      __syncthreads();
      if (threadIdx.x == 0 && d.gctr >= 0) {   // every thread's stores precede the barrier
        __threadfence();
        atomicAdd(gdone + d.gctr, 1);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ solves
// Right-hand side of a slab solve: either a raw slab field, or the gather of
// global columns (ga, gb] plus the transmission injections of SubdomSolve
// (Table 2) at the local columns ef (tau1, from B1) and eb (tau3, from B3).
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
  int bnr, br0;               // transmission buffers: [2][bnr][ny], this launch's rhs from br0
};

// Epilogue of a slab solve (Table 2): the slab solution's core columns into
// the global field and the two layers passed on by the transmission.
template <typename R>
struct Out {
  cplx<R>* raw;               // [n_rhs][ny][W] or null
  cplx<R>* u;                 // global field [n_rhs][ny][nx]: columns (ua, ub] are stored
  int nx, lo, wl, ua, ub;     // (each sweep phase writes every column exactly once)
  cplx<R>* B2;                // [2][n_rhs][ny]: layers at local e2, e2+1 (tau2)
  int e2;
  cplx<R>* B4;                // layers at local e4, e4+1 (tau4)
  int e4;
  int bnr, br0;               // as in Rhs
};

template <typename R>
struct SolveArgs {
  int W, wp, ny, nr;
  int P, S0, mid;             // segments (the first S0 on the top chain), meeting row
  const int4* seg;            // per segment: first row, rows, direction (+1 top, -1 bottom), group
  int NG, G0;                 // segment groups (the first G0 on the top chain)
  const int4* grp;            // per group: first segment, last segment, half, index in the half
  const cplx<R>* Phi;         // [P][mstride] segment transfer products (forward)
  const cplx<R>* Psi;         //   (backward)
  const cplx<R>* PhiP;        // [P][mstride] their in-group prefix products
  const cplx<R>* PsiP;
  const cplx<R>* st;          // [ny][9][wp]
  const cplx<R>* G;           // [ny][gstride]: G_k = S_k^-1
  const cplx<R>* F;           // [ny][mstride]: F'_k = G_k L_k (coupling to the previous chain row)
  const cplx<R>* E;           // [ny][mstride]: E'_k = G_k R_k (coupling to the next chain row)
  size_t gstride;             // elements per G block (W x W)
  size_t mstride;             // elements per F', E', Phi, Psi block (W rows of stride wp)
  int stages;
  cplx<R>* Y;                 // [ny][nr][wp]: G_k f_k, then forward rows y_k
  cplx<R>* carry_f;           // [P+NG][nr][wp]: segment end values of the forward recurrence
                              //   (in-group values, zero group start); [P+g]: group g's true end
  cplx<R>* carry_b;           // [P+1+NG][nr][wp]: segment start values of the backward one
                              //   (in-group); [P]: x_m; [P+1+g]: group g's true start
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
    const cplx<R>* B = q.B1 + ((size_t)(1 - s) * q.bnr + q.br0 + r) * ny;
    for (int dy = -1; dy <= 1; ++dy) {
      int kk = k + dy;
      if (kk >= 0 && kk < ny) cfma(v, c[dy + 1], B[kk]);
    }
  }
  if (q.eb >= 0 && (e == q.eb || e == q.eb + 1)) {
    int s = e - q.eb;
    const cplx<R>* c = q.inj + ((size_t)(2 + s) * ny + k) * 3;
    const cplx<R>* B = q.B3 + ((size_t)(1 - s) * q.bnr + q.br0 + r) * ny;
    for (int dy = -1; dy <= 1; ++dy) {
      int kk = k + dy;
      if (kk >= 0 && kk < ny) cfma(v, c[dy + 1], B[kk]);
    }
  }
  return v;
}

// Pipeline stage: [matrix (gstride) | vector row (nr wp)].
template <typename R>
struct Pipe {
  uint64_t* bar;
  cplx<R>* buf;
  int stages;
  size_t stage_elems, gstride;
  int wp, nr;
  __device__ cplx<R>* slot(int i) const { return buf + (size_t)i * stage_elems; }
  // thread 0 only: fetch the matrix of block row k and, if `rows` is given,
  // the vector row k of rows
  __device__ void issue(int i, int k, const cplx<R>* M, const cplx<R>* rows) const {
    const uint32_t mb = (uint32_t)(gstride * sizeof(cplx<R>));
    const uint32_t vb = rows ? (uint32_t)((size_t)nr * wp * sizeof(cplx<R>)) : 0u;
    cplx<R>* dst = slot(i);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[i], mb + vb);
    tma_load_1d(dst, M + (size_t)k * gstride, mb, &bar[i]);
    if (rows) tma_load_1d(dst + gstride, rows + (size_t)k * nr * wp, vb, &bar[i]);
  }
  // The same in two halves: the matrix (written before the solve began, so
  // it may be fetched before pdl_wait) and, after pdl_wait, the vector row
  // with the stage's arrival.
  __device__ void issue_matrix(int i, int k, const cplx<R>* M) const {
    const uint32_t mb = (uint32_t)(gstride * sizeof(cplx<R>));
    mbar_expect_tx_noarrive(&bar[i], mb);
    tma_load_1d(slot(i), M + (size_t)k * gstride, mb, &bar[i]);
  }
  __device__ void issue_vector(int i, int k, const cplx<R>* rows) const {
    const uint32_t vb = (uint32_t)((size_t)nr * wp * sizeof(cplx<R>));
    mbar_expect_tx(&bar[i], vb);
    tma_load_1d(slot(i) + gstride, rows + (size_t)k * nr * wp, vb, &bar[i]);
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

// gemv_rows for matrices and vectors of row stride ldm = ldv = wp (wp = 4 mod
// 8, zero beyond W): complex64 entries are read in pairs (128-bit loads).
// With wp = 4 mod 8 the eight rows a warp reads at once fall on disjoint
// bank groups, so every load takes the minimum number of wavefronts.
template <typename R, int NR>
__device__ __forceinline__ void gemv_op(const cplx<R>* M, int ldm, const cplx<R>* v, int ldv,
                                        int W, int nr, int row, int lane, cplx<R> (&acc)[NR]) {
  if constexpr (sizeof(R) == 4) {
    float ar[NR], ai[NR], br[NR], bi[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) { ar[r] = 0.f; ai[r] = 0.f; br[r] = 0.f; bi[r] = 0.f; }
    if (row < W) {
      const float4* Mr = reinterpret_cast<const float4*>(M + (size_t)row * ldm);
      const int npair = ldm >> 1;
      for (int p = lane; p < npair; p += kTPR) {
        const float4 m = Mr[p];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          const float4 x = reinterpret_cast<const float4*>(v + (size_t)r * ldv)[p];
          ar[r] += m.x * x.x - m.y * x.y;
          ai[r] += m.x * x.y + m.y * x.x;
          br[r] += m.z * x.z - m.w * x.w;
          bi[r] += m.z * x.w + m.w * x.z;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      acc[r] = mk<R>(ar[r] + br[r], ai[r] + bi[r]);
#pragma unroll
      for (int o = kTPR / 2; o > 0; o >>= 1) {
        acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, o);
        acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, o);
      }
    }
  } else {
    gemv_rows<R, NR>(M, ldm, v, ldv, W, nr, row, lane, acc);
  }
}

// Shared memory of the substitution kernels: barriers, two NR x wp vectors
// (the recurrence value, double-buffered so that a step needs one block
// barrier), then the pipeline stages.
template <typename R>
__device__ __forceinline__ void init_pipe(Pipe<R>& pipe, unsigned char* smem, const SolveArgs<R>& a,
                                          int NR, cplx<R>** vec) {
  pipe.bar = (uint64_t*)smem;
  *vec = (cplx<R>*)(smem + 128);
  cplx<R>* b = *vec + 2 * NR * a.wp;
  pipe.buf = (cplx<R>*)(((uintptr_t)b + 127) & ~(uintptr_t)127);
  pipe.stages = a.stages;
  pipe.gstride = a.mstride;
  pipe.wp = a.wp;
  pipe.nr = a.nr;
  pipe.stage_elems = a.mstride + (size_t)a.nr * a.wp;
}

// SubdomSolve (Table 2): the slab right-hand side (gather + transmission
// injection) of block row k, premultiplied by its factor block: Y[k] =
// G_k f_k (the meeting row keeps f_m).  One CTA per block row; every row is
// independent.  G_k comes into shared memory by one bulk copy, issued before
// pdl_wait (the factors are written before the solve begins); the gather
// reads the predecessor's results after it.
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_rhs_kernel(SolveArgs<R> a) {
  const int k = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, nr = a.nr;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  const int grp = tid / kTPR, lane = tid % kTPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  uint64_t* bar = (uint64_t*)smem_raw;
  cplx<R>* f = (cplx<R>*)(smem_raw + 128);   // NR x wp
  cplx<R>* Gs = (cplx<R>*)(((uintptr_t)(f + NR * wp) + 127) & ~(uintptr_t)127);
  const bool mid = (k == a.mid);
  const uint32_t gb = (uint32_t)(a.gstride * sizeof(cplx<R>));
  if (tid == 0) {
    sh_abort = 0;
    mbar_init(bar, 1);
    mbar_fence_init();
    if (!mid) {
      mbar_expect_tx(bar, gb);
      tma_load_1d(Gs, a.G + (size_t)k * a.gstride, gb, bar);
    }
  }
  pdl_trigger();
  pdl_wait();
  for (int i = tid; i < NR * wp; i += nthr) {
    const int r = i / wp, e = i - r * wp;
    f[i] = (r < nr && e < W) ? rhs_at<R>(a.rhs, a.ny, W, nr, r, k, e) : mk<R>(0, 0);
  }
  __syncthreads();
  cplx<R>* Yk = a.Y + (size_t)k * nr * wp;
  if (mid) {
    for (int i = tid; i < nr * wp; i += nthr) Yk[i] = f[i];
    return;
  }
  if (!mbar_wait(bar, 0, a.flag)) sh_abort = 1;
  __syncthreads();
  if (sh_abort) return;
  cplx<R> acc[NR];
  for (int rb = 0; rb < W; rb += ngroups) {
    const int row = rb + grp;
    gemv_rows<R, NR>(Gs, W, f, wp, W, nr, row, lane, acc);
    if (lane == 0 && row < W)
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < nr) Yk[r * wp + row] = acc[r];
  }
  if (tid < nr * (wp - W)) {            // padding columns
    const int r = tid / (wp - W), e = W + tid % (wp - W);
    Yk[r * wp + e] = mk<R>(0, 0);
  }
}

// Forward recurrence over segment s along its chain, t = 0..n-1, rows
// k_t = k0 + dir t:  y_t = g_t - F'_t y_{t-1}  (g_t = G_t f_t, F'_t = G_t L_t).
//   mode 0: zero start, store only the last y into carry_f[s];
//   mode 1: start from the true end value of segment s-1 (zero for the
//           first segment of each half), store every y into Y (over g); if
//           bwd1, then run the
//           backward recurrence x_t = y_t - E'_t x_{t+1} (E'_t = G_t R_t)
//           over the segment from a zero start and store x_0 into carry_b[s].
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_fwd_kernel(SolveArgs<R> a, int mode, int bwd1) {
  const int s = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, nr = a.nr;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  const int4 sd = a.seg[s];
  const int k0 = sd.x, n = sd.y, dir = sd.z;
  const bool first = (s == 0 || s == a.S0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  Pipe<R> pipe;
  cplx<R>* vec;
  init_pipe<R>(pipe, smem_raw, a, NR, &vec);
  const int VS = NR * wp;
  const cplx<R> zero = mk<R>(0, 0);
  // Start value (mode 1): the true end y of segment q = s-1.  In the first
  // group of a half the in-group values are true; otherwise one fix-up step
  // y_q = carry_f[q] + PhiP_q y_in (y_in: the previous group's true end)
  // runs as pipeline item 0, ahead of the rows.
  const int q = s - 1;
  int fix = 0;
  const cplx<R>* vin = nullptr;
  if (mode == 1 && !first) {
    const int gi = a.seg[q].w;
    if (gi == (s >= a.S0 ? a.G0 : 0)) {
      vin = a.carry_f + (size_t)q * nr * wp;
    } else {
      fix = 1;
      vin = a.carry_f + (size_t)(a.P + gi - 1) * nr * wp;
    }
  }
  const int nit = n + fix;
  auto issue_item = [&](int slot, int it) {
    if (it < fix) pipe.issue(slot, q, a.PhiP, a.carry_f);
    else pipe.issue(slot, k0 + dir * (it - fix), a.F, a.Y);
  };
  // the operator blocks of the first stages before the predecessor ends
  const int npre = min(pipe.stages, nit);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
    for (int i = 0; i < npre; ++i) {
      if (i < fix) pipe.issue_matrix(i, q, a.PhiP);
      else pipe.issue_matrix(i, k0 + dir * (i - fix), a.F);
    }
  }
  pdl_trigger();
  pdl_wait();
  // both buffers in full: the paired loads of the GEMV also read the padding
  for (int i = tid; i < 2 * VS; i += nthr) {
    const int r = i / wp, e = i - r * wp;
    vec[i] = (i < VS && vin && r < nr && e < W) ? vin[r * wp + e] : zero;
  }
  if (tid == 0)
    for (int i = 0; i < npre; ++i) {
      if (i < fix) pipe.issue_vector(i, q, a.carry_f);
      else pipe.issue_vector(i, k0 + dir * (i - fix), a.Y);
    }
  __syncthreads();
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  int cur = 0;
  for (int it = 0; it < nit; ++it) {
    const bool fx = it < fix;
    const int k = k0 + dir * (it - fix);
    const int slot = it % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Mk = pipe.slot(slot);
    const cplx<R>* gk = Mk + pipe.gstride;
    const cplx<R>* yp = vec + cur * VS;
    cplx<R>* yn = vec + (cur ^ 1) * VS;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_op<R, NR>(Mk, wp, yp, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          const cplx<R> y = fx ? gk[r * wp + row] + acc[r] : gk[r * wp + row] - acc[r];
          yn[r * wp + row] = y;
          if (mode == 1 && !fx) a.Y[((size_t)k * nr + r) * wp + row] = y;
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    cur ^= 1;
    if (tid == 0 && it + pipe.stages < nit) issue_item(slot, it + pipe.stages);
  }
  if (mode == 0) {
    for (int i = tid; i < nr * wp; i += nthr) a.carry_f[(size_t)s * nr * wp + i] = vec[cur * VS + i];
    return;
  }
  if (!bwd1) return;
  // Backward recurrence from a zero start.  The y rows were written above by
  // this CTA (generic stores); they are read with ordinary loads, one step
  // ahead, never through TMA; the pipeline brings only E'_t.
  for (int i = tid; i < VS; i += nthr) vec[cur * VS + i] = zero;   // x_n
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i)
      pipe.issue(i, k0 + dir * (n - 1 - i), a.E, nullptr);
  cplx<R> ynext[NR];
  {
    const int row0 = grp;   // rows handled by this group in the first pass over rb
    const int kl = k0 + dir * (n - 1);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      ynext[r] = (lane == 0 && row0 < W && r < nr) ? a.Y[((size_t)kl * nr + r) * wp + row0] : zero;
  }
  for (int q = 0; q < n; ++q) {
    const int t = n - 1 - q;
    const int k = k0 + dir * t;
    const int slot = q % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Mk = pipe.slot(slot);
    const cplx<R>* xp = vec + cur * VS;
    cplx<R>* xn = vec + (cur ^ 1) * VS;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      cplx<R> ycur[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) ycur[r] = ynext[r];
      if (rb + ngroups >= W) {           // last pass over rows: prefetch the next row
        const int rowp = grp;
#pragma unroll
        for (int r = 0; r < NR; ++r)
          ynext[r] = (lane == 0 && rowp < W && r < nr && t > 0)
                         ? a.Y[((size_t)(k - dir) * nr + r) * wp + rowp] : zero;
      }
      if (rb > 0) {                      // rows beyond the first pass: plain load now
#pragma unroll
        for (int r = 0; r < NR; ++r)
          ycur[r] = (lane == 0 && row < W && r < nr) ? a.Y[((size_t)k * nr + r) * wp + row] : zero;
      }
      gemv_op<R, NR>(Mk, wp, xp, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          xn[r * wp + row] = ycur[r] - acc[r];
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    cur ^= 1;
    if (tid == 0 && q + pipe.stages < n) pipe.issue(slot, k - dir * pipe.stages, a.E, nullptr);
  }
  for (int i = tid; i < nr * wp; i += nthr) a.carry_b[(size_t)s * nr * wp + i] = vec[cur * VS + i];
}

// Epilogue of Table 2 for one solution entry x at block row k, local column row.
template <typename R>
__device__ __forceinline__ void store_out(const Out<R>& o, int ny, int W, int nr, int r, int k,
                                          int row, cplx<R> x) {
  const int g = row - o.wl + o.lo;
  if (o.raw) o.raw[((size_t)r * ny + k) * W + row] = x;
  if (o.u && g > o.ua && g <= o.ub) o.u[((size_t)r * ny + k) * o.nx + g] = x;
  if (o.B2 && (row == o.e2 || row == o.e2 + 1))
    o.B2[((size_t)(row - o.e2) * o.bnr + o.br0 + r) * ny + k] = x;
  if (o.B4 && (row == o.e4 || row == o.e4 + 1))
    o.B4[((size_t)(row - o.e4) * o.bnr + o.br0 + r) * ny + k] = x;
}

// Final backward recurrence over segment s from x_{n} = the true start value
// of segment s+1 (last segment of a half: the meeting row's x_m = carry_b[P]),
// with the epilogue of Table 2.
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_bwd_kernel(SolveArgs<R> a) {
  const int s = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, ny = a.ny, nr = a.nr;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  const int4 sd = a.seg[s];
  const int k0 = sd.x, n = sd.y, dir = sd.z;
  const bool last = (s == a.S0 - 1 || s == a.P - 1);
  // Start value: x_m after the last segment of a half; otherwise the true
  // start of segment q = s+1 by one fix-up step x_q = carry_b[q] + PsiP_q x_in
  // (pipeline item 0; x_in: the true start of the next group towards the
  // meeting row, or x_m).
  const int q = s + 1;
  const int fix = last ? 0 : 1;
  const cplx<R>* vin = a.carry_b + (size_t)a.P * nr * wp;
  if (!last) {
    const int gi = a.seg[q].w;
    const int glast = s >= a.S0 ? a.NG - 1 : a.G0 - 1;
    if (gi != glast) vin = a.carry_b + (size_t)(a.P + 2 + gi) * nr * wp;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  Pipe<R> pipe;
  cplx<R>* vec;
  init_pipe<R>(pipe, smem_raw, a, NR, &vec);
  const int VS = NR * wp;
  const cplx<R> zero = mk<R>(0, 0);
  const int nit = n + fix;
  auto issue_item = [&](int slot, int it) {
    if (it < fix) pipe.issue(slot, q, a.PsiP, a.carry_b);
    else pipe.issue(slot, k0 + dir * (n - 1 - (it - fix)), a.E, a.Y);
  };
  const int npre = min(pipe.stages, nit);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
    for (int i = 0; i < npre; ++i) {
      if (i < fix) pipe.issue_matrix(i, q, a.PsiP);
      else pipe.issue_matrix(i, k0 + dir * (n - 1 - (i - fix)), a.E);
    }
  }
  pdl_trigger();
  pdl_wait();
  for (int i = tid; i < 2 * VS; i += nthr) {   // both buffers (padding is read)
    const int r = i / wp, e = i - r * wp;
    vec[i] = (i < VS && r < nr && e < W) ? vin[r * wp + e] : zero;
  }
  if (tid == 0)
    for (int i = 0; i < npre; ++i) {
      if (i < fix) pipe.issue_vector(i, q, a.carry_b);
      else pipe.issue_vector(i, k0 + dir * (n - 1 - (i - fix)), a.Y);
    }
  __syncthreads();
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  int cur = 0;
  for (int it = 0; it < nit; ++it) {
    const bool fx = it < fix;
    const int k = k0 + dir * (n - 1 - (it - fix));
    const int slot = it % pipe.stages;
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Mk = pipe.slot(slot);
    const cplx<R>* yk = Mk + pipe.gstride;
    const cplx<R>* xp = vec + cur * VS;
    cplx<R>* xn = vec + (cur ^ 1) * VS;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_op<R, NR>(Mk, wp, xp, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          const cplx<R> x = fx ? yk[r * wp + row] + acc[r] : yk[r * wp + row] - acc[r];
          xn[r * wp + row] = x;
          if (!fx) store_out<R>(a.out, ny, W, nr, r, k, row, x);
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    cur ^= 1;
    if (tid == 0 && it + pipe.stages < nit) issue_item(slot, it + pipe.stages);
  }
}

// Two-level segment carries.  Every kind runs the recurrence
//   v_i = hat_i + M_i v_{i-1}
// over a list of segments through a TMA pipeline (stage = [M_i | hat row]),
// the running value double-buffered:
//   kind 0 (forward, one CTA per group): segments q_lo+1 .. q_hi from
//          v = carry_f[q_lo] (zero group start), M = Phi_q; the in-group
//          values replace yhat in carry_f[q];
//   kind 1 (backward, one CTA per group): q_hi-1 .. q_lo from carry_b[q_hi],
//          M = Psi_q, in carry_b[q];
//   kind 2 (forward, one CTA per half): the half's groups g = 1, 2, ... from
//          the first group's end (its in-group values are true), M = PhiP of
//          the group's last segment, hat = its in-group value; v = the
//          group's true end, stored in carry_f[P+g];
//   kind 3 (backward, one CTA per half): first the meeting row
//          x_m = G_m (f_m - C_m y_{m-1} - B_m y_{m+1}) (stored in carry_b[P] and
//          the output by the first CTA), then the half's groups from the
//          meeting row outwards, M = PsiP of the group's first segment; v =
//          the group's true start, stored in carry_b[P+1+g].
template <typename R, int NR>
__global__ void __launch_bounds__(kThreads) slab_carry_kernel(SolveArgs<R> a, int kind) {
  const int b = blockIdx.x, tid = threadIdx.x, W = a.W, wp = a.wp, nr = a.nr, P = a.P;
  const int nthr = blockDim.x, ngroups = nthr / kTPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  uint64_t* bar = (uint64_t*)smem_raw;
  cplx<R>* prev = (cplx<R>*)(smem_raw + 128);   // 2 x NR x wp
  const int VS = NR * wp;
  cplx<R>* vtmp = prev + 2 * VS;
  cplx<R>* buf = (cplx<R>*)(((uintptr_t)(vtmp + VS) + 127) & ~(uintptr_t)127);
  const size_t se = a.mstride + (size_t)nr * wp;
  const size_t RW = (size_t)nr * wp;            // elements per carry row
  const int stages = a.stages;
  const bool bwd = (kind & 1) != 0;
  cplx<R>* carry = bwd ? a.carry_b : a.carry_f;
  const cplx<R>* prod = kind == 0 ? a.Phi : kind == 1 ? a.Psi : kind == 2 ? a.PhiP : a.PsiP;
  const uint32_t mb = (uint32_t)(a.mstride * sizeof(cplx<R>));
  const uint32_t vb = (uint32_t)(RW * sizeof(cplx<R>));
  int4 gr = make_int4(0, 0, 0, 0);
  int g_first = 0, ng = 0, nsteps;
  if (kind < 2) {
    gr = a.grp[b];
    nsteps = gr.y - gr.x;
  } else {
    g_first = b ? a.G0 : 0;
    ng = b ? a.NG - a.G0 : a.G0;
    nsteps = kind == 2 ? ng - 1 : ng;
  }
  // segment (product and hat row) of step i, and the row its result goes to
  auto seg_of = [&](int i) -> int {
    if (kind == 0) return gr.x + 1 + i;
    if (kind == 1) return gr.y - 1 - i;
    if (kind == 2) return a.grp[g_first + 1 + i].y;
    return a.grp[g_first + ng - 1 - i].x;
  };
  auto out_row = [&](int i) -> size_t {
    if (kind == 0) return (size_t)(gr.x + 1 + i);
    if (kind == 1) return (size_t)(gr.y - 1 - i);
    if (kind == 2) return (size_t)(P + g_first + 1 + i);
    return (size_t)(P + 1 + g_first + ng - 1 - i);
  };
  auto issue = [&](int slot, int i) {
    const int sg = seg_of(i);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[slot], mb + vb);
    tma_load_1d(buf + (size_t)slot * se, prod + (size_t)sg * a.mstride, mb, &bar[slot]);
    tma_load_1d(buf + (size_t)slot * se + a.mstride, carry + (size_t)sg * RW, vb, &bar[slot]);
  };
  const cplx<R> zero = mk<R>(0, 0);
  // the products of the first stages before the predecessor ends; their
  // hat rows (written by the predecessor) after pdl_wait
  const int npre = min(stages, nsteps);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < stages; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
    for (int i = 0; i < npre; ++i) {
      mbar_expect_tx_noarrive(&bar[i], mb);
      tma_load_1d(buf + (size_t)i * se, prod + (size_t)seg_of(i) * a.mstride, mb, &bar[i]);
    }
  }
  pdl_trigger();
  pdl_wait();
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[NR];
  for (int i = tid; i < 2 * VS; i += nthr) prev[i] = zero;   // both buffers (padding is read)
  if (kind >= 2) {   // the group-boundary rows in full (zero padding)
    for (int i = tid; i < nsteps * (int)RW; i += nthr) {
      const int st = i / (int)RW, e = i % wp;
      if (e >= W) carry[out_row(st) * RW + i % RW] = zero;
    }
  }
  __syncthreads();
  if (kind < 3) {
    const size_t srow = kind == 0 ? gr.x : kind == 1 ? gr.y : a.grp[g_first].y;
    for (int i = tid; i < (int)RW; i += nthr) {
      const cplx<R> v = (i % wp < W) ? carry[srow * RW + i] : zero;
      prev[i] = v;
      if (kind == 2) carry[(size_t)(P + g_first) * RW + i] = v;
    }
  } else {
    // meeting row: v = f_m - C_m y_{m-1} - B_m y_{m+1}, x_m = G_m v; y_{m-1}
    // and y_{m+1} are the true ends of the last groups of the two halves
    const int m = a.mid;
    const cplx<R>* stm = a.st + (size_t)m * 9 * wp;
    const cplx<R>* yu = a.carry_f + (size_t)(P + a.G0 - 1) * RW;
    const cplx<R>* yd = a.carry_f + (size_t)(P + a.NG - 1) * RW;
    for (int i = tid; i < VS; i += nthr) {
      const int r = i / wp, e = i - r * wp;
      cplx<R> v = zero;
      if (r < nr && e < W) {
        v = a.Y[((size_t)m * nr + r) * wp + e];
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int ee = e + dx;
          if (ee < 0 || ee >= W) continue;
          v = v - stm[(dx + 1) * wp + e] * yu[r * wp + ee] - stm[(6 + dx + 1) * wp + e] * yd[r * wp + ee];
        }
      }
      vtmp[i] = v;
    }
    __syncthreads();
    const cplx<R>* Gm = a.G + (size_t)m * a.gstride;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_rows<R, NR>(Gm, W, vtmp, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W)
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r < nr) {
            prev[r * wp + row] = acc[r];
            if (b == 0) store_out<R>(a.out, a.ny, W, nr, r, m, row, acc[r]);
          }
    }
    __syncthreads();
    if (b == 0)   // the whole row, zero padding included
      for (int i = tid; i < (int)RW; i += nthr) a.carry_b[(size_t)P * RW + i] = prev[i];
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < npre; ++i) {
      mbar_expect_tx(&bar[i], vb);
      tma_load_1d(buf + (size_t)i * se + a.mstride, carry + (size_t)seg_of(i) * RW, vb, &bar[i]);
    }
  uint32_t phase_bits = 0;
  int cur = 0;
  for (int i = 0; i < nsteps; ++i) {
    const size_t orow = out_row(i);
    const int slot = i % stages;
    if (!mbar_wait(&bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* M = buf + (size_t)slot * se;
    const cplx<R>* hat = M + a.mstride;
    const cplx<R>* pp = prev + cur * VS;
    cplx<R>* pn = prev + (cur ^ 1) * VS;
    for (int rb = 0; rb < W; rb += ngroups) {
      const int row = rb + grp;
      gemv_op<R, NR>(M, wp, pp, wp, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nr) break;
          const cplx<R> res = hat[r * wp + row] + acc[r];
          pn[r * wp + row] = res;
          carry[orow * RW + r * wp + row] = res;
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    cur ^= 1;
    if (tid == 0 && i + stages < nsteps) issue(slot, i + stages);
  }
}

// ------------------------------------------------------------------ host side
template <typename R>
static size_t solve_smem(const Slab& S, int nr, int NR, int stages) {
  const size_t el = sizeof(cplx<R>);
  size_t fixed = 128 + 2 * (size_t)NR * S.wp * el + 128;
  size_t stage = (S.mstride + (size_t)nr * S.wp) * el;
  return fixed + (size_t)stages * stage;
}

template <typename R>
static size_t carry_smem(const Slab& S, int nr, int NR, int stages) {
  const size_t el = sizeof(cplx<R>);
  return 128 + 3 * (size_t)NR * S.wp * el + 128 + (size_t)stages * (S.mstride + (size_t)nr * S.wp) * el;
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
  const int J = L.J, P = L.P, m = L.mid;
  constexpr int BW = FactorPanel<R>::BW;
  const size_t el = sizeof(cplx<R>);
  int maxW = 0;
  for (int j = 1; j <= J; ++j) maxW = std::max(maxW, L.slabs[j].W);
  const size_t smem_f = factor_smem_bytes(maxW, 18, el, BW);
  const size_t smem_m = factor_smem_bytes(maxW, 15, el, BW);
  // products: M, T, the couplings and, when it fits, A_t
  const size_t smem_p2 = (2 * (size_t)maxW * maxW + 3 * (size_t)maxW) * el;
  const int stage_a = smem_p2 + (size_t)maxW * maxW * el <= kSmemLimit ? 1 : 0;
  const size_t smem_p = smem_p2 + (stage_a ? (size_t)maxW * maxW * el : 0);
  // delayed updates: rows per update warp (RPW) and columns per lane (CPL);
  // register tiles of the product GEMMs: 4 x 4 while they fit, else 4 x 8
  // (the 12 main update warps take RPW rows each; at most 3 rows are left to
  // the three late warps)
  const int rpw = std::max(1, (maxW - kLateUpdateWarps + kMainUpdateWarps - 1) / kMainUpdateWarps);
  if (maxW > 128 || rpw > 11 || smem_m > kSmemLimit || smem_p > kSmemLimit ||
      2 * (size_t)maxW * maxW * el > kSmemLimit)
    throw Failure(HZ_EINVAL, "slab too wide for the blocked factorisation (W=" +
                                 std::to_string(maxW) + ")");
  std::vector<FactorDesc> fd;
  std::vector<MidDesc> md;
  std::vector<ProdDesc> pd, pf;   // product tasks; prefix tasks of the fused launch
  std::vector<PrefixDesc> xd;     // prefix tasks of the separate launch
  const int NG = L.NG;
  // group completion counter of slab j, direction bwd (0: Phi, 1: Psi), group g
  auto gctr = [&](int j, int bwd, int g) { return ((j - 1) * 2 + bwd) * NG + g; };
  for (int j = 1; j <= J; ++j) {
    const Slab& S = L.slabs[j];
    const int dg = L.fe ? 0 : 1;   // finite differences: 5-point, diagonal couplings
    fd.push_back(FactorDesc{S.W, S.wp, 0, m, +1, dg, S.st, S.G, S.gstride});
    fd.push_back(FactorDesc{S.W, S.wp, L.ny - 1, L.ny - 1 - m, -1, dg, S.st, S.G, S.gstride});
    md.push_back(MidDesc{S.W, S.wp, m, S.st, S.G, S.gstride});
    for (int q = 0; q < P; ++q) {
      const int4 sg = L.seg[q];
      // (Phi of the first segment of a half is never used: operators only)
      // rows of the segment are final once its chain has passed them
      const int fchain = 2 * (j - 1) + (sg.z > 0 ? 0 : 1);
      const int need = (sg.z > 0 ? sg.x : L.ny - 1 - sg.x) + sg.y;
      pd.push_back(ProdDesc{S.W, S.wp, sg.x, sg.y, sg.z, 0, (q != 0 && q != L.S0) ? 1 : 0,
                            stage_a, fchain, need, S.st, S.G, S.F, S.gstride, S.mstride,
                            (cplx<R>*)S.Phi + (size_t)q * S.mstride, 0, gctr(j, 0, sg.w), 0});
      pd.push_back(ProdDesc{S.W, S.wp, sg.x, sg.y, sg.z, 1, 1, stage_a, fchain, need, S.st, S.G,
                            S.E, S.gstride, S.mstride, (cplx<R>*)S.Psi + (size_t)q * S.mstride, 0,
                            gctr(j, 1, sg.w), 0});
    }
    // in-group prefix products: forward for every group but the first of a
    // half (whose in-group values are already true), backward for all; a
    // group is complete once the chain has finished its last segment
    for (int gi = 0; gi < NG; ++gi) {
      const int4 g = L.grp[gi];
      const int n = g.y - g.x + 1;
      const int4 last = L.seg[g.y];
      const int fchain = 2 * (j - 1) + (last.z > 0 ? 0 : 1);
      const int need = (last.z > 0 ? last.x : L.ny - 1 - last.x) + last.y;
      if (g.w != 0) {
        xd.push_back(PrefixDesc{S.W, S.wp, g.x, n, +1, S.Phi, S.PhiP, S.mstride});
        pf.push_back(ProdDesc{S.W, S.wp, g.x, n, +1, 0, 0, 0, fchain, need, nullptr, nullptr,
                              S.Phi, 0, S.mstride, S.PhiP, 1, gctr(j, 0, gi), n});
      }
      xd.push_back(PrefixDesc{S.W, S.wp, g.y, n, -1, S.Psi, S.PsiP, S.mstride});
      pf.push_back(ProdDesc{S.W, S.wp, g.y, n, -1, 1, 0, 0, fchain, need, nullptr, nullptr, S.Psi,
                            0, S.mstride, S.PsiP, 1, gctr(j, 1, gi), n});
    }
  }
  // tasks in the order their rows become final; a prefix task after every
  // product task of its group (equal needs: products first)
  auto by_need = [](const ProdDesc& x, const ProdDesc& y) { return x.need < y.need; };
  std::stable_sort(pd.begin(), pd.end(), by_need);
  std::vector<ProdDesc> pdx(pd);
  pdx.insert(pdx.end(), pf.begin(), pf.end());
  std::stable_sort(pdx.begin(), pdx.end(), by_need);
  const size_t b_fd = sizeof(FactorDesc) * fd.size(), b_md = sizeof(MidDesc) * md.size();
  const size_t b_pd = sizeof(ProdDesc) * pd.size(), b_xd = sizeof(PrefixDesc) * xd.size();
  const size_t b_pdx = sizeof(ProdDesc) * pdx.size();
  // chain progress [nf], task counter [1], group completion counters [2 J NG]
  const size_t nsync = fd.size() + 1 + (size_t)2 * J * NG;
  // The descriptors depend only on the slab geometry and buffers, which are
  // fixed from set-up on: they are uploaded by the first factorisation of
  // the level and kept (with the sync counters) until the level is freed,
  // so later factorisations allocate nothing.
  if (!L.fac_desc) {
    L.fac_desc = dmalloc(b_fd + b_md + b_pd + b_xd + b_pdx);
    L.fac_sync = (int*)dmalloc(sizeof(int) * nsync);
    unsigned char* d = (unsigned char*)L.fac_desc;
    HZ_CU(cudaMemcpyAsync(d, fd.data(), b_fd, cudaMemcpyHostToDevice, s));
    HZ_CU(cudaMemcpyAsync(d + b_fd, md.data(), b_md, cudaMemcpyHostToDevice, s));
    HZ_CU(cudaMemcpyAsync(d + b_fd + b_md, pd.data(), b_pd, cudaMemcpyHostToDevice, s));
    HZ_CU(cudaMemcpyAsync(d + b_fd + b_md + b_pd, xd.data(), b_xd, cudaMemcpyHostToDevice, s));
    HZ_CU(cudaMemcpyAsync(d + b_fd + b_md + b_pd + b_xd, pdx.data(), b_pdx,
                          cudaMemcpyHostToDevice, s));
  }
  unsigned char* d_desc = (unsigned char*)L.fac_desc;
  FactorDesc* d_fd = (FactorDesc*)d_desc;
  MidDesc* d_md = (MidDesc*)(d_desc + b_fd);
  ProdDesc* d_pd = (ProdDesc*)(d_desc + b_fd + b_md);
  PrefixDesc* d_xd = (PrefixDesc*)(d_desc + b_fd + b_md + b_pd);
  ProdDesc* d_pdx = (ProdDesc*)(d_desc + b_fd + b_md + b_pd + b_xd);
  int* d_sync = L.fac_sync;
  HZ_CU(cudaMemsetAsync(d_sync, 0, sizeof(int) * nsync, s));
  int coop = 0;
  HZ_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev));
  if (test_hook("HZ_TEST_NO_COOP") > 0) coop = 0;        // exercises the separate launches
  const long long hook_ns = test_hook("HZ_TEST_WAIT_LIMIT_NS");
  const unsigned long long wait_ns = hook_ns >= 0 ? (unsigned long long)hook_ns : 10000000000ull;
  const size_t smem_x = 2 * (size_t)maxW * maxW * el;   // prefix products: M, T
  auto run = [&](auto kf, auto km, auto kp, auto kfused, auto kx) {
    HZ_CU(cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m));
    // one cooperative launch: the chains and, beside them on the other SMs,
    // the product tasks as their rows become final
    const size_t smem_u = std::max(smem_f, smem_p);
    HZ_CU(cudaFuncSetAttribute(kfused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u));
    int per_sm = 0;
    HZ_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfused, kThreads, smem_u));
    const long resident = (long)per_sm * h->sms;
    const int nf = (int)fd.size(), np = (int)pd.size(), npx = (int)pdx.size();
    const bool fused = coop && resident > nf;
    if (fused) {
      const unsigned grid = (unsigned)std::min<long>(resident, (long)nf + npx);
      const FactorDesc* a0 = d_fd;
      const ProdDesc* a2 = d_pdx;
      int* a4 = d_sync;
      int* a5 = d_sync + nf;
      int* a6 = d_sync + nf + 1;
      int* a7 = h->dev_flag;
      unsigned long long a8 = wait_ns;
      void* args[] = {(void*)&a0, (void*)&nf, (void*)&a2, (void*)&npx, (void*)&a4, (void*)&a5,
                      (void*)&a6, (void*)&a7, (void*)&a8};
      timed(h, "slab_factor", 0.0, s, [&] {
        HZ_CU(cudaLaunchCooperativeKernel((const void*)kfused, dim3(grid), dim3(kThreads), args,
                                          smem_u, s));
      });
      h->launches += 1;
    } else {
      HZ_CU(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f));
      HZ_CU(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
      timed(h, "slab_factor", 0.0, s, [&] { kf<<<(unsigned)nf, kThreads, smem_f, s>>>(d_fd); });
      timed(h, "segment_product", 0.0, s,
            [&] { kp<<<(unsigned)np, kThreads, smem_p, s>>>(d_pd); });
      h->launches += 2;
    }
    timed(h, "slab_middle", 0.0, s, [&] { km<<<(unsigned)md.size(), kThreads, smem_m, s>>>(d_md); });
    h->launches += 1;
    if (!fused) {   // (inside the fused launch otherwise)
      HZ_CU(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x));
      timed(h, "segment_prefix", 0.0, s,
            [&] { kx<<<(unsigned)xd.size(), kThreads, smem_x, s>>>(d_xd); });
      h->launches += 1;
    }
  };
  // factor: update strips (RPW rows, CPL columns per lane); product GEMMs:
  // 16 warps x PRPW rows, PCPL columns per lane
  auto with_prod = [&](auto kf, auto km, auto tag_rpw, auto tag_cpl) {
    constexpr int FR = decltype(tag_rpw)::value, FC = decltype(tag_cpl)::value;
    if (maxW <= 64)
      run(kf, km, segment_product_kernel<R, 4, 2>, slab_factor_fused_kernel<R, FR, FC, 4, 2>,
          segment_prefix_kernel<R, 4, 2>);
    else if (maxW <= 80)
      run(kf, km, segment_product_kernel<R, 5, 3>, slab_factor_fused_kernel<R, FR, FC, 5, 3>,
          segment_prefix_kernel<R, 5, 3>);
    else if (maxW <= 96)
      run(kf, km, segment_product_kernel<R, 6, 3>, slab_factor_fused_kernel<R, FR, FC, 6, 3>,
          segment_prefix_kernel<R, 6, 3>);
    else
      run(kf, km, segment_product_kernel<R, 8, 4>, slab_factor_fused_kernel<R, FR, FC, 8, 4>,
          segment_prefix_kernel<R, 8, 4>);
  };
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  using I5 = std::integral_constant<int, 5>;
  using I6 = std::integral_constant<int, 6>;
  using I8 = std::integral_constant<int, 8>;
  using I11 = std::integral_constant<int, 11>;
  if (maxW <= 64) {
    if (rpw <= 4) with_prod(slab_factor_kernel<R, 4, 2>, slab_middle_kernel<R, 4, 2>, I4{}, I2{});
    else with_prod(slab_factor_kernel<R, 5, 2>, slab_middle_kernel<R, 5, 2>, I5{}, I2{});
  } else if (maxW <= 96) {
    if (rpw <= 6) with_prod(slab_factor_kernel<R, 6, 3>, slab_middle_kernel<R, 6, 3>, I6{}, I3{});
    else with_prod(slab_factor_kernel<R, 8, 3>, slab_middle_kernel<R, 8, 3>, I8{}, I3{});
  } else {
    with_prod(slab_factor_kernel<R, 11, 4>, slab_middle_kernel<R, 11, 4>, I11{}, I4{});
  }
  HZ_CU(cudaGetLastError());
  HZ_CU(cudaStreamSynchronize(s));
}

template <typename R, int NR>
static void set_solve_attrs() {
  static bool done = false;
  if (done) return;
  HZ_CU(cudaFuncSetAttribute(slab_fwd_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  HZ_CU(cudaFuncSetAttribute(slab_bwd_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  HZ_CU(cudaFuncSetAttribute(slab_carry_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  HZ_CU(cudaFuncSetAttribute(slab_rhs_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  done = true;
}

// Launch with programmatic stream serialisation: the kernel may start while
// its predecessor in the stream runs; it fetches only data written before the
// solve began until pdl_wait() (every kernel launched this way calls it
// before touching its predecessor's results).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
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

// Launch sequence of one slab solve; `tagged` brackets the kernels with
// timing events (when timing is on).  All eight kernels overlap their
// prologues with their predecessors (programmatic dependent launch).
template <typename R, int NR>
static void launch_solve(hz_handle* h, Level& L, Slab& S, SolveArgs<R> a, cudaStream_t s,
                         bool tagged) {
  set_solve_attrs<R, NR>();
  const int P = L.P, nr = a.nr;
  a.stages = pick_stages<R>(S, nr, NR);
  // more segments than SMs: shallower pipelines, so that two segment CTAs
  // share an SM and every segment pass stays one wave
  if (P > h->sms)
    while (a.stages > 1 && solve_smem<R>(S, nr, NR, a.stages) > (size_t)110 * 1024) --a.stages;
  const size_t smem = solve_smem<R>(S, nr, NR, a.stages);
  const double el = sizeof(cplx<R>);
  const double gbytes = (double)L.ny * S.W * S.W * el;          // one pass over G_0..G_{ny-1}
  const double vbytes = (double)nr * L.ny * S.W * el;           // one slab-sized vector
  const double lbytes = (double)(P - L.NG) * S.W * S.W * el;   // in-group carry products
  const double bbytes = (double)L.NG * S.W * S.W * el;          // group-boundary products
  auto T = [&](const char* tag, double bytes, auto&& fn) {
    if (tagged) timed(h, tag, bytes, s, fn); else fn();
  };
  // one 4-thread group per row of G: round W * kTPR up to whole warps
  const int nthr = std::min(kThreads, std::max(128, (S.W * kTPR + 31) / 32 * 32));
  SolveArgs<R> ac = a;
  ac.stages = pick_carry_stages<R>(S, nr, NR);
  const size_t csm = carry_smem<R>(S, nr, NR, ac.stages);
  const size_t rsmem = 256 + ((size_t)NR * S.wp + S.gstride) * sizeof(cplx<R>);
  T("slab_rhs", gbytes + 2 * vbytes,
    [&] { launch_pdl(slab_rhs_kernel<R, NR>, L.ny, (unsigned)nthr, rsmem, s, a); });
  const unsigned nt = (unsigned)nthr;
  T("slab_fwd_pass1", gbytes + vbytes,
    [&] { launch_pdl(slab_fwd_kernel<R, NR>, P, nt, smem, s, a, 0, 0); });
  T("slab_carry", lbytes, [&] { launch_pdl(slab_carry_kernel<R, NR>, L.NG, nt, csm, s, ac, 0); });
  T("slab_carry_bound", bbytes, [&] { launch_pdl(slab_carry_kernel<R, NR>, 2, nt, csm, s, ac, 2); });
  T("slab_fwd_bwd1", 2 * gbytes + 3 * vbytes,
    [&] { launch_pdl(slab_fwd_kernel<R, NR>, P, nt, smem, s, a, 1, 1); });
  T("slab_carry", lbytes, [&] { launch_pdl(slab_carry_kernel<R, NR>, L.NG, nt, csm, s, ac, 1); });
  T("slab_carry_bound", bbytes, [&] { launch_pdl(slab_carry_kernel<R, NR>, 2, nt, csm, s, ac, 3); });
  T("slab_bwd", gbytes + 2 * vbytes, [&] { launch_pdl(slab_bwd_kernel<R, NR>, P, nt, smem, s, a); });
  h->launches += 8;
  HZ_CU(cudaGetLastError());
}

template <typename R>
static void run_solve(hz_handle* h, Level& L, Slab& S, const Rhs<R>& rhs, const Out<R>& out,
                      int n_rhs, cudaStream_t s, cplx<R>* Y, cplx<R>* cf, cplx<R>* cb,
                      bool tagged) {
  if (n_rhs > kNRMax) {       // chunks of at most kNRMax right-hand sides
    for (int r0 = 0; r0 < n_rhs; r0 += kNRMax) {
      const int nr = std::min(kNRMax, n_rhs - r0);
      Rhs<R> q = rhs;
      Out<R> o = out;
      q.bnr = o.bnr = n_rhs;
      q.br0 = o.br0 = r0;
      const size_t in_f = (size_t)L.ny * L.nx, in_raw = (size_t)L.ny * S.W;
      if (q.raw) q.raw += r0 * in_raw;
      if (q.f) q.f += r0 * in_f;
      if (o.raw) o.raw += r0 * in_raw;
      if (o.u) o.u += r0 * in_f;
      run_solve<R>(h, L, S, q, o, nr, s, Y, cf, cb, tagged);
    }
    return;
  }
  if (n_rhs < 1) throw Failure(HZ_EINVAL, "right-hand sides per slab launch must be >= 1");
  SolveArgs<R> a;
  a.W = S.W; a.wp = S.wp; a.ny = L.ny; a.nr = n_rhs;
  a.F = (const cplx<R>*)S.F; a.E = (const cplx<R>*)S.E; a.mstride = S.mstride;
  a.P = L.P; a.S0 = L.S0; a.mid = L.mid; a.seg = L.seg_dev;
  a.NG = L.NG; a.G0 = L.G0; a.grp = L.grp_dev;
  a.Phi = (const cplx<R>*)S.Phi; a.Psi = (const cplx<R>*)S.Psi;
  a.PhiP = (const cplx<R>*)S.PhiP; a.PsiP = (const cplx<R>*)S.PsiP;
  a.st = (const cplx<R>*)S.st; a.G = (const cplx<R>*)S.G; a.gstride = S.gstride;
  a.stages = 1;
  a.Y = Y; a.carry_f = cf; a.carry_b = cb;
  a.flag = h->dev_flag;
  a.rhs = rhs;
  a.out = out;
  if (a.rhs.bnr == 0) a.rhs.bnr = n_rhs;    // one launch for all right-hand sides
  if (a.out.bnr == 0) a.out.bnr = n_rhs;
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
// (Y [ny][n_rhs][wp], segment carries [P+NG] and [P+1+NG] rows of n_rhs x wp); the same kernels
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

}  // namespace hz
