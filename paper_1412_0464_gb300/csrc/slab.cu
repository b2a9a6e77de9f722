// Slab factorisation and slab solves (the subdomain solves of SubdomSolve,
// Table 2; the paper uses a sparse direct solver, Section 5).
//
// A^(j) is block tridiagonal along y with W x W blocks (one block row per
// grid row k): D_k couples row k to itself, C_k to row k-1, B_k to row k+1
// (taken from the slab stencil st[k][9][W]).  Block LU:
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
__device__ __forceinline__ void fence_proxy_async() {
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
constexpr int kNR = 8;                  // right-hand sides per launch

// --------------------------------------------------------------- factorisation
struct FactorDesc {
  int W, ny;
  const void* st;
  void* G;
  size_t gstride;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) slab_factor_kernel(const FactorDesc* descs) {
  const FactorDesc d = descs[blockIdx.x];
  const int W = d.W, ny = d.ny, tid = threadIdx.x;
  const cplx<R>* st = (const cplx<R>*)d.st;
  cplx<R>* G = (cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* S = (cplx<R>*)smem_raw;          // W*W
  cplx<R>* T = S + W * W;                   // W*W
  cplx<R>* colp = T + W * W;                // W
  int* perm = (int*)(colp + W);             // W
  __shared__ int sh_r;
  __shared__ cplx<R> sh_inv;
  const cplx<R> zero = mk<R>(0, 0);
  for (int k = 0; k < ny; ++k) {
    const cplx<R>* stk = st + (size_t)k * 9 * W;
    if (k == 0) {
      for (int i = tid; i < W * W; i += kThreads) S[i] = zero;
    } else {
      // T = G_{k-1} B_{k-1}: T[a][b] = sum_dx G[a][b-dx] * B_{k-1}(b-dx, dx)
      const cplx<R>* stp = st + (size_t)(k - 1) * 9 * W;
      for (int i = tid; i < W * W; i += kThreads) {
        int a = i / W, b = i - a * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          int e = b - dx;
          if (e >= 0 && e < W) cfma(acc, S[a * W + e], stp[(6 + dx + 1) * W + e]);
        }
        T[i] = acc;
      }
      __syncthreads();
      // S = -C_k T: S[a][b] = -sum_dx C_k(a, dx) T[a+dx][b]
      for (int i = tid; i < W * W; i += kThreads) {
        int a = i / W, b = i - a * W;
        cplx<R> acc = zero;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          int e = a + dx;
          if (e >= 0 && e < W) cfma(acc, stk[(0 + dx + 1) * W + a], T[e * W + b]);
        }
        S[i] = -acc;
      }
    }
    __syncthreads();
    // + D_k
    for (int a = tid; a < W; a += kThreads) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int b = a + dx;
        if (b >= 0 && b < W) S[a * W + b] = S[a * W + b] + stk[(3 + dx + 1) * W + a];
      }
    }
    __syncthreads();
    // In-place Gauss-Jordan inversion with partial pivoting.
    for (int p = 0; p < W; ++p) {
      if (tid < 32) {
        R best = -1;
        int bi = p;
        for (int i = p + tid; i < W; i += 32) {
          R v = cabs2(S[i * W + p]);
          if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          R ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) { sh_r = bi; perm[p] = bi; }
      }
      __syncthreads();
      const int r = sh_r;
      if (r != p) {
        for (int j = tid; j < W; j += kThreads) {
          cplx<R> t = S[p * W + j];
          S[p * W + j] = S[r * W + j];
          S[r * W + j] = t;
        }
        __syncthreads();
      }
      for (int i = tid; i < W; i += kThreads) colp[i] = S[i * W + p];
      if (tid == 0) sh_inv = cinv(S[p * W + p]);
      __syncthreads();
      const cplx<R> inv = sh_inv;
      for (int j = tid; j < W; j += kThreads) S[p * W + j] = (j == p ? mk<R>(1, 0) : S[p * W + j]) * inv;
      __syncthreads();
      for (int i = tid; i < W * W; i += kThreads) {
        int a = i / W, b = i - a * W;
        if (a == p) continue;
        cplx<R> v = (b == p) ? zero : S[i];
        cplx<R> c = colp[a];
        cplx<R> q = S[p * W + b];
        v.re -= c.re * q.re - c.im * q.im;
        v.im -= c.re * q.im + c.im * q.re;
        S[i] = v;
      }
      __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int p = W - 1; p >= 0; --p) {
      int r = perm[p];
      if (r != p) {
        for (int i = tid; i < W; i += kThreads) {
          cplx<R> t = S[i * W + p];
          S[i * W + p] = S[i * W + r];
          S[i * W + r] = t;
        }
        __syncthreads();
      }
    }
    cplx<R>* Gk = G + (size_t)k * d.gstride;
    for (int i = tid; i < W * W; i += kThreads) Gk[i] = S[i];
    __syncthreads();
  }
}

// ------------------------------------------------------------ segment products
struct ProdDesc {
  int W, k0, k1, backward;
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
  const int W = d.W, tid = threadIdx.x;
  const cplx<R>* st = (const cplx<R>*)d.st;
  const cplx<R>* G = (const cplx<R>*)d.G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* M = (cplx<R>*)smem_raw;
  cplx<R>* T = M + W * W;
  const cplx<R> zero = mk<R>(0, 0);
  for (int i = tid; i < W * W; i += kThreads) M[i] = (i / W == i % W) ? mk<R>(1, 0) : zero;
  __syncthreads();
  const int n = d.k1 - d.k0;
  const int plane = d.backward ? 6 : 0;   // B_k (dy=+1) or C_k (dy=-1)
  for (int s = 0; s < n; ++s) {
    const int k = d.backward ? d.k1 - 1 - s : d.k0 + s;
    const cplx<R>* stk = st + (size_t)k * 9 * W;
    for (int i = tid; i < W * W; i += kThreads) {      // T = coupling_k M
      int a = i / W, c = i - a * W;
      cplx<R> acc = zero;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int e = a + dx;
        if (e >= 0 && e < W) cfma(acc, stk[(plane + dx + 1) * W + a], M[e * W + c]);
      }
      T[i] = acc;
    }
    __syncthreads();
    const cplx<R>* Gk = G + (size_t)k * d.gstride;
    for (int i = tid; i < W * W; i += kThreads) {      // M = -G_k T
      int a = i / W, c = i - a * W;
      cplx<R> acc = zero;
      for (int j = 0; j < W; ++j) cfma(acc, Gk[a * W + j], T[j * W + c]);
      M[i] = -acc;
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
  cplx<R>* u;                 // global field [n_rhs][ny][nx]
  int nx, lo, wl, ua, ub;     // scatter global columns (ua, ub]
  cplx<R>* B2;                // [2][n_rhs][ny]: layers at local e2, e2+1 (tau2)
  int e2;
  cplx<R>* B4;                // layers at local e4, e4+1 (tau4)
  int e4;
};

template <typename R>
struct SolveArgs {
  int W, ny, n_rhs, P;
  const int* seg;
  const cplx<R>* st;
  const cplx<R>* G;
  size_t gstride;
  int stages;
  cplx<R>* Y;                 // [n_rhs][ny][W]
  cplx<R>* carry_f;           // [P][n_rhs][W]
  cplx<R>* carry_b;
  int* flag;
  Rhs<R> rhs;
  Out<R> out;
};

template <typename R>
__device__ __forceinline__ cplx<R> rhs_at(const Rhs<R>& q, int ny, int W, int nr, int r, int k, int e) {
  const cplx<R> zero = mk<R>(0, 0);
  if (q.raw) return q.raw[((size_t)r * ny + k) * W + e];
  cplx<R> v = zero;
  int g = e - q.wl + q.lo;
  if (g > q.ga && g <= q.gb) v = q.f[((size_t)r * ny + k) * q.nx + g];
  if (q.ef >= 0 && (e == q.ef || e == q.ef + 1)) {
    int s = e - q.ef;                          // 0: row beta uses B[1]; 1: row beta+1 uses B[0]
    const cplx<R>* c = q.inj + ((size_t)s * ny + k) * 3;
    const cplx<R>* B = q.B1 + ((size_t)(1 - s) * nr + r) * ny;  // layer 1-s
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

// Shared-memory pipeline of G blocks (one TMA bulk copy per block row).
template <typename R>
struct GPipe {
  uint64_t* bar;
  cplx<R>* buf;
  int stages;
  uint32_t bytes;
  const cplx<R>* G;
  size_t gstride;
  __device__ cplx<R>* slot(int i) { return buf + (size_t)i * gstride; }
  __device__ void issue(int i, int k) {     // thread 0 only
    fence_proxy_async();
    mbar_expect_tx(&bar[i], bytes);
    tma_load_1d(slot(i), G + (size_t)k * gstride, bytes, &bar[i]);
  }
};

// y = M v for NR right-hand sides, M row-major W x W in shared memory; the
// TPR threads of a group split the columns and reduce with shuffles.
// Called by every thread of the block with the same trip count; rows >= W
// contribute zeros so that the shuffles stay warp-uniform.
template <typename R>
__device__ __forceinline__ void gemv_rows(const cplx<R>* M, const cplx<R>* v, int W, int nr,
                                          int row, int lane, cplx<R>* acc) {
  for (int r = 0; r < kNR; ++r) acc[r] = mk<R>(0, 0);
  const cplx<R>* Mr = M + (size_t)row * W;
  const int jend = row < W ? W : 0;
  for (int j = lane; j < jend; j += kTPR) {
    cplx<R> m = Mr[j];
#pragma unroll
    for (int r = 0; r < kNR; ++r)
      if (r < nr) cfma(acc[r], m, v[r * W + j]);
  }
#pragma unroll
  for (int r = 0; r < kNR; ++r) {
    if (r < nr) {
#pragma unroll
      for (int o = kTPR / 2; o > 0; o >>= 1) {
        acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, o);
        acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, o);
      }
    }
  }
}

// Forward recurrence over one segment.
//   mode 0: zero start, store only the segment's last y into carry_f[p];
//   mode 1: start from carry_f[p-1] (segment 0: zero), store every y_k into Y;
//           if bwd1, then run the backward recurrence over the segment from a
//           zero start and store its first x into carry_b[p].
template <typename R>
__global__ void __launch_bounds__(kThreads) slab_fwd_kernel(SolveArgs<R> a, int mode, int bwd1) {
  const int p = blockIdx.x, tid = threadIdx.x, W = a.W, ny = a.ny, nr = a.n_rhs;
  const int k0 = a.seg[p], k1 = a.seg[p + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  GPipe<R> pipe;
  pipe.bar = (uint64_t*)smem_raw;
  cplx<R>* vbuf = (cplx<R>*)(smem_raw + 128);
  cplx<R>* ybuf = vbuf + kNR * W;
  pipe.buf = ybuf + kNR * W;
  pipe.buf = (cplx<R>*)(((uintptr_t)pipe.buf + 127) & ~(uintptr_t)127);
  pipe.stages = a.stages;
  pipe.bytes = (uint32_t)(a.gstride * sizeof(cplx<R>));
  pipe.G = a.G;
  pipe.gstride = a.gstride;
  const cplx<R> zero = mk<R>(0, 0);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
  }
  // initial y_{k0-1}
  for (int i = tid; i < nr * W; i += kThreads) {
    int r = i / W, e = i - r * W;
    ybuf[i] = (mode == 1 && p > 0) ? a.carry_f[((size_t)(p - 1) * nr + r) * W + e] : zero;
  }
  __syncthreads();
  const int n = k1 - k0;
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k0 + i);
  uint32_t phase_bits = 0;   // parity per stage
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[kNR];
  for (int s = 0; s < n; ++s) {
    const int k = k0 + s;
    const cplx<R>* stk = a.st + (size_t)k * 9 * W;
    // v_k = f_k - C_k y_{k-1}
    for (int i = tid; i < nr * W; i += kThreads) {
      int r = i / W, e = i - r * W;
      cplx<R> v = rhs_at<R>(a.rhs, ny, W, nr, r, k, e);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int ee = e + dx;
        if (ee >= 0 && ee < W) {
          cplx<R> c = stk[(0 + dx + 1) * W + e];
          cplx<R> y = ybuf[r * W + ee];
          v.re -= c.re * y.re - c.im * y.im;
          v.im -= c.re * y.im + c.im * y.re;
        }
      }
      vbuf[i] = v;
    }
    const int slot = s % pipe.stages;
    __syncthreads();
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    for (int rb = 0; rb < W; rb += kGroups) {
      const int row = rb + grp;
      gemv_rows<R>(Gk, vbuf, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
        for (int r = 0; r < nr; ++r) {
          ybuf[r * W + row] = acc[r];
          if (mode == 1) a.Y[((size_t)r * ny + k) * W + row] = acc[r];
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k + pipe.stages);
  }
  if (mode == 0) {
    for (int i = tid; i < nr * W; i += kThreads) {
      int r = i / W, e = i - r * W;
      a.carry_f[((size_t)p * nr + r) * W + e] = ybuf[i];
    }
    return;
  }
  if (!bwd1) return;
  // backward recurrence from a zero start: x_k = y_k - G_k (B_k x_{k+1})
  for (int i = tid; i < nr * W; i += kThreads) ybuf[i] = zero;  // x_{k1}
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k1 - 1 - i);
  // stage parities continue from the forward pass: each stage was used a
  // known number of times; phase_bits already tracks them.
  for (int s = 0; s < n; ++s) {
    const int k = k1 - 1 - s;
    const cplx<R>* stk = a.st + (size_t)k * 9 * W;
    for (int i = tid; i < nr * W; i += kThreads) {      // w = B_k x_{k+1}
      int r = i / W, e = i - r * W;
      cplx<R> v = zero;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int ee = e + dx;
        if (ee >= 0 && ee < W) cfma(v, stk[(6 + dx + 1) * W + e], ybuf[r * W + ee]);
      }
      vbuf[i] = v;
    }
    const int slot = s % pipe.stages;
    __syncthreads();
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    for (int rb = 0; rb < W; rb += kGroups) {
      const int row = rb + grp;
      gemv_rows<R>(Gk, vbuf, W, nr, row, lane, acc);
      if (lane == 0 && row < W)
        for (int r = 0; r < nr; ++r) ybuf[r * W + row] = a.Y[((size_t)r * ny + k) * W + row] - acc[r];
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k - pipe.stages);
  }
  for (int i = tid; i < nr * W; i += kThreads) {
    int r = i / W, e = i - r * W;
    a.carry_b[((size_t)p * nr + r) * W + e] = ybuf[i];
  }
}

// Final backward recurrence over one segment from x_{k1} = carry_b[p+1]
// (last segment: zero), with the epilogue of Table 2.
template <typename R>
__global__ void __launch_bounds__(kThreads) slab_bwd_kernel(SolveArgs<R> a) {
  const int p = blockIdx.x, tid = threadIdx.x, W = a.W, ny = a.ny, nr = a.n_rhs;
  const int k0 = a.seg[p], k1 = a.seg[p + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh_abort;
  GPipe<R> pipe;
  pipe.bar = (uint64_t*)smem_raw;
  cplx<R>* vbuf = (cplx<R>*)(smem_raw + 128);
  cplx<R>* xbuf = vbuf + kNR * W;
  pipe.buf = xbuf + kNR * W;
  pipe.buf = (cplx<R>*)(((uintptr_t)pipe.buf + 127) & ~(uintptr_t)127);
  pipe.stages = a.stages;
  pipe.bytes = (uint32_t)(a.gstride * sizeof(cplx<R>));
  pipe.G = a.G;
  pipe.gstride = a.gstride;
  const cplx<R> zero = mk<R>(0, 0);
  if (tid == 0) {
    sh_abort = 0;
    for (int i = 0; i < pipe.stages; ++i) mbar_init(&pipe.bar[i], 1);
    mbar_fence_init();
  }
  for (int i = tid; i < nr * W; i += kThreads) {
    int r = i / W, e = i - r * W;
    xbuf[i] = (p + 1 < a.P) ? a.carry_b[((size_t)(p + 1) * nr + r) * W + e] : zero;
  }
  __syncthreads();
  const int n = k1 - k0;
  if (tid == 0)
    for (int i = 0; i < pipe.stages && i < n; ++i) pipe.issue(i, k1 - 1 - i);
  uint32_t phase_bits = 0;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[kNR];
  const Out<R>& o = a.out;
  for (int s = 0; s < n; ++s) {
    const int k = k1 - 1 - s;
    const cplx<R>* stk = a.st + (size_t)k * 9 * W;
    for (int i = tid; i < nr * W; i += kThreads) {
      int r = i / W, e = i - r * W;
      cplx<R> v = zero;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int ee = e + dx;
        if (ee >= 0 && ee < W) cfma(v, stk[(6 + dx + 1) * W + e], xbuf[r * W + ee]);
      }
      vbuf[i] = v;
    }
    const int slot = s % pipe.stages;
    __syncthreads();
    if (!mbar_wait(&pipe.bar[slot], (phase_bits >> slot) & 1u, a.flag)) sh_abort = 1;
    phase_bits ^= 1u << slot;
    const cplx<R>* Gk = pipe.slot(slot);
    for (int rb = 0; rb < W; rb += kGroups) {
      const int row = rb + grp;
      gemv_rows<R>(Gk, vbuf, W, nr, row, lane, acc);
      if (lane == 0 && row < W) {
        const int g = row - o.wl + o.lo;
        for (int r = 0; r < nr; ++r) {
          cplx<R> x = a.Y[((size_t)r * ny + k) * W + row] - acc[r];
          xbuf[r * W + row] = x;
          if (o.raw) o.raw[((size_t)r * ny + k) * W + row] = x;
          if (o.u && g > o.ua && g <= o.ub) {
            cplx<R>* uu = o.u + ((size_t)r * ny + k) * o.nx + g;
            *uu = *uu + x;
          }
          if (o.B2 && (row == o.e2 || row == o.e2 + 1))
            o.B2[((size_t)(row - o.e2) * nr + r) * ny + k] = x;
          if (o.B4 && (row == o.e4 || row == o.e4 + 1))
            o.B4[((size_t)(row - o.e4) * nr + r) * ny + k] = x;
        }
      }
    }
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0 && s + pipe.stages < n) pipe.issue(slot, k - pipe.stages);
  }
}

// Segment carries: forward Y_p = yhat_p + Phi_p Y_{p-1}; backward
// X_p = xhat_p + Psi_p X_{p+1}.
template <typename R>
__global__ void __launch_bounds__(kThreads) slab_carry_kernel(SolveArgs<R> a, const cplx<R>* prod,
                                                              int backward) {
  const int tid = threadIdx.x, W = a.W, nr = a.n_rhs, P = a.P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* prev = (cplx<R>*)smem_raw;  // [nr][W]
  cplx<R>* nxt = prev + kNR * W;       // [nr][W]
  cplx<R>* carry = backward ? a.carry_b : a.carry_f;
  const int grp = tid / kTPR, lane = tid % kTPR;
  cplx<R> acc[kNR];
  const int pstart = backward ? P - 1 : 0;
  for (int i = tid; i < nr * W; i += kThreads) prev[i] = carry[(size_t)pstart * nr * W + i];
  __syncthreads();
  for (int q = 1; q < P; ++q) {
    const int p = backward ? P - 1 - q : q;
    const cplx<R>* M = prod + (size_t)p * a.gstride;
    cplx<R>* cp = carry + (size_t)p * nr * W;
    for (int rb = 0; rb < W; rb += kGroups) {
      const int row = rb + grp;
      gemv_rows<R>(M, prev, W, nr, row, lane, acc);
      if (lane == 0 && row < W)
        for (int r = 0; r < nr; ++r) nxt[r * W + row] = cp[r * W + row] + acc[r];
    }
    __syncthreads();
    for (int i = tid; i < nr * W; i += kThreads) {
      cp[i] = nxt[i];
      prev[i] = nxt[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host side
static size_t solve_smem(int W, size_t gstride, size_t elem, int stages) {
  size_t fixed = 128 + 2 * kNR * (size_t)W * elem + 128;
  return fixed + (size_t)stages * gstride * elem;
}

template <typename R>
static int pick_stages(const Slab& S) {
  const size_t limit = 225 * 1024;
  int st = 4;
  while (st > 1 && solve_smem(S.W, S.gstride, sizeof(cplx<R>), st) > limit) --st;
  if (solve_smem(S.W, S.gstride, sizeof(cplx<R>), st) > limit)
    throw Failure(HZ_EINVAL, "slab too wide for the shared-memory slab solve (W=" +
                                 std::to_string(S.W) + ")");
  return st;
}

template <typename R>
void factor_level(hz_handle* h, Level& L, cudaStream_t s) {
  const int J = L.J;
  int maxW = 0;
  for (int j = 1; j <= J; ++j) maxW = std::max(maxW, L.slabs[j].W);
  size_t smem = 2 * (size_t)maxW * maxW * sizeof(cplx<R>) + maxW * (sizeof(cplx<R>) + sizeof(int)) + 64;
  if (smem > 225 * 1024)
    throw Failure(HZ_EINVAL, "slab too wide for the shared-memory factorisation (W=" +
                                 std::to_string(maxW) + ")");
  std::vector<FactorDesc> fd(J);
  for (int j = 1; j <= J; ++j) {
    const Slab& S = L.slabs[j];
    fd[j - 1] = FactorDesc{S.W, L.ny, S.st, S.G, S.gstride};
  }
  FactorDesc* d_fd = (FactorDesc*)dmalloc(sizeof(FactorDesc) * J);
  HZ_CU(cudaMemcpyAsync(d_fd, fd.data(), sizeof(FactorDesc) * J, cudaMemcpyHostToDevice, s));
  HZ_CU(cudaFuncSetAttribute(slab_factor_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
  slab_factor_kernel<R><<<J, kThreads, smem, s>>>(d_fd);
  h->launches++;
  HZ_CU(cudaGetLastError());
  ProdDesc* d_pd = nullptr;
  if (L.P > 1) {
    std::vector<ProdDesc> pd;
    for (int j = 1; j <= J; ++j) {
      const Slab& S = L.slabs[j];
      for (int p = 0; p < L.P; ++p)
        for (int bw = 0; bw < 2; ++bw)
          pd.push_back(ProdDesc{S.W, L.seg[p], L.seg[p + 1], bw, S.st, S.G, S.gstride,
                                (cplx<R>*)(bw ? S.Psi : S.Phi) + (size_t)p * S.gstride});
    }
    d_pd = (ProdDesc*)dmalloc(sizeof(ProdDesc) * pd.size());
    HZ_CU(cudaMemcpyAsync(d_pd, pd.data(), sizeof(ProdDesc) * pd.size(), cudaMemcpyHostToDevice, s));
    size_t psm = 2 * (size_t)maxW * maxW * sizeof(cplx<R>);
    HZ_CU(cudaFuncSetAttribute(segment_product_kernel<R>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    segment_product_kernel<R><<<(unsigned)pd.size(), kThreads, psm, s>>>(d_pd);
    h->launches++;
    HZ_CU(cudaGetLastError());
  }
  HZ_CU(cudaStreamSynchronize(s));
  dfree(d_fd);
  dfree(d_pd);
}

template <typename R>
static void run_solve(hz_handle* h, Level& L, Slab& S, const Rhs<R>& rhs, const Out<R>& out,
                      int n_rhs, cudaStream_t s) {
  if (n_rhs > kNR) throw Failure(HZ_EINVAL, "too many right-hand sides per slab launch");
  SolveArgs<R> a;
  a.W = S.W; a.ny = L.ny; a.n_rhs = n_rhs; a.P = L.P; a.seg = L.seg_dev;
  a.st = (const cplx<R>*)S.st; a.G = (const cplx<R>*)S.G; a.gstride = S.gstride;
  a.stages = pick_stages<R>(S);
  a.Y = (cplx<R>*)S.Y; a.carry_f = (cplx<R>*)S.carry_f; a.carry_b = (cplx<R>*)S.carry_b;
  a.flag = h->dev_flag;
  a.rhs = rhs;
  a.out = out;
  size_t smem = solve_smem(S.W, S.gstride, sizeof(cplx<R>), a.stages);
  static bool attr_set[2] = {false, false};
  int ai = sizeof(R) == 8 ? 1 : 0;
  if (!attr_set[ai]) {
    HZ_CU(cudaFuncSetAttribute(slab_fwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    HZ_CU(cudaFuncSetAttribute(slab_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    attr_set[ai] = true;
  }
  const int P = L.P;
  const double el = sizeof(cplx<R>);
  const double gbytes = (double)L.ny * S.W * S.W * el;          // one pass over G_0..G_{ny-1}
  const double vbytes = (double)n_rhs * L.ny * S.W * el;        // one slab-sized vector
  const double pbytes = (double)P * S.W * S.W * el;             // one set of segment products
  dim3 grid(P);
  auto seq = [&] {
    if (P == 1) {
      timed(h, "slab_fwd", gbytes + 2 * vbytes, s, [&] {
        slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 1, 0);
      });
      timed(h, "slab_bwd", gbytes + 2 * vbytes, s, [&] {
        slab_bwd_kernel<R><<<grid, kThreads, smem, s>>>(a);
      });
      h->launches += 2;
    } else {
      size_t csm = 2 * (size_t)kNR * S.W * sizeof(cplx<R>);
      timed(h, "slab_fwd_pass1", gbytes + vbytes, s, [&] {
        slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 0, 0);
      });
      timed(h, "slab_carry", pbytes, s, [&] {
        slab_carry_kernel<R><<<1, kThreads, csm, s>>>(a, (const cplx<R>*)S.Phi, 0);
      });
      timed(h, "slab_fwd_bwd1", 2 * gbytes + 3 * vbytes, s, [&] {
        slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 1, 1);
      });
      timed(h, "slab_carry", pbytes, s, [&] {
        slab_carry_kernel<R><<<1, kThreads, csm, s>>>(a, (const cplx<R>*)S.Psi, 1);
      });
      timed(h, "slab_bwd", gbytes + 2 * vbytes, s, [&] {
        slab_bwd_kernel<R><<<grid, kThreads, smem, s>>>(a);
      });
      h->launches += 5;
    }
  };
  // the whole slab solve; algorithmic bytes = the method's minimum: G read
  // once per substitution direction plus right-hand side and solution
  timed(h, "slab_solve", 2 * gbytes + 2 * vbytes, s, seq);
  HZ_CU(cudaGetLastError());
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
  run_solve<R>(h, L, S, q, o, n_rhs, s);
}

template <typename R>
void slab_solve_raw(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud, int n_rhs,
                    cudaStream_t s) {
  Slab& S = L.slabs[j];
  Rhs<R> q{};
  q.raw = fd; q.ef = -1; q.eb = -1;
  Out<R> o{};
  o.raw = ud; o.e2 = -1; o.e4 = -1;
  run_solve<R>(h, L, S, q, o, n_rhs, s);
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

}  // namespace hz

namespace hz {

// Slab solve of a raw right-hand side with caller-provided work buffers
// (forward-solution rows Y [n_rhs][ny][W] and segment carries
// [P][n_rhs][W] each); launches the same kernels as slab_solve_raw and
// allocates nothing.
template <typename R>
void slab_solve_raw_scratch(hz_handle* h, Level& L, int j, const cplx<R>* fd, cplx<R>* ud,
                            int n_rhs, cudaStream_t s, cplx<R>* Y, cplx<R>* carry_f,
                            cplx<R>* carry_b) {
  Slab& S = L.slabs[j];
  if (n_rhs > kNR) throw Failure(HZ_EINVAL, "too many right-hand sides per slab launch");
  SolveArgs<R> a;
  a.W = S.W; a.ny = L.ny; a.n_rhs = n_rhs; a.P = L.P; a.seg = L.seg_dev;
  a.st = (const cplx<R>*)S.st; a.G = (const cplx<R>*)S.G; a.gstride = S.gstride;
  a.stages = pick_stages<R>(S);
  a.Y = Y; a.carry_f = carry_f; a.carry_b = carry_b;
  a.flag = h->dev_flag;
  a.rhs = Rhs<R>{};
  a.rhs.raw = fd; a.rhs.ef = -1; a.rhs.eb = -1;
  a.out = Out<R>{};
  a.out.raw = ud; a.out.e2 = -1; a.out.e4 = -1;
  const size_t smem = solve_smem(S.W, S.gstride, sizeof(cplx<R>), a.stages);
  HZ_CU(cudaFuncSetAttribute(slab_fwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
  HZ_CU(cudaFuncSetAttribute(slab_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
  const int P = L.P;
  dim3 grid(P);
  if (P == 1) {
    slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 1, 0);
    slab_bwd_kernel<R><<<grid, kThreads, smem, s>>>(a);
    h->launches += 2;
  } else {
    const size_t csm = 2 * (size_t)kNR * S.W * sizeof(cplx<R>);
    slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 0, 0);
    slab_carry_kernel<R><<<1, kThreads, csm, s>>>(a, (const cplx<R>*)S.Phi, 0);
    slab_fwd_kernel<R><<<grid, kThreads, smem, s>>>(a, 1, 1);
    slab_carry_kernel<R><<<1, kThreads, csm, s>>>(a, (const cplx<R>*)S.Psi, 1);
    slab_bwd_kernel<R><<<grid, kThreads, smem, s>>>(a);
    h->launches += 5;
  }
  HZ_CU(cudaGetLastError());
}

template void slab_solve_raw_scratch<float>(hz_handle*, Level&, int, const c64*, c64*, int,
                                            cudaStream_t, c64*, c64*, c64*);
template void slab_solve_raw_scratch<double>(hz_handle*, Level&, int, const c128*, c128*, int,
                                             cudaStream_t, c128*, c128*, c128*);

}  // namespace hz
