/*
 * hz.h -- C ABI of the GB300 sweeping-preconditioner Helmholtz solver.
 *
 * Method: C. C. Stolk, "An improved sweeping domain decomposition
 * preconditioner for the Helmholtz equation" (arXiv 1412.0464).  The library
 * solves the discretised Helmholtz equation with PML truncation (Section 2.1,
 * Eqs. 3-5; discretisation Eq. 40) by restarted GMRES preconditioned by the
 * double-sweep domain decomposition with PML transmission (Section 2.2,
 * Tables 2-3), optionally inside the two-grid sweeping preconditioner
 * (Section 4, Appendix A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  A rectangle (2-D) or box (3-D).  Along axis l there are n[l]
 *   interior cells of size h and w_out PML cells on each side:
 *   n[l] + 2 w_out cells and N_l = n[l] + 2 w_out - 1 unknowns (Dirichlet
 *   nodes on the outer boundary, Section 2.2).  x (l = 0) is the sweep axis;
 *   n_dof = prod_l N_l and N_t = n_dof / N_x (the transverse unknowns).
 * Layout.  Fields are dense, contiguous, [rhs][y][x] (2-D) or [rhs][z][y][x]
 *   (3-D), x fastest.  Complex values are interleaved (re, im) doubles.
 * System.  A is Eq. 40 multiplied by h^d (complex symmetric; in 3-D the
 *   7-point analogue, each second difference divided by the PML factors of
 *   the other two axes).  The right-hand side b of A u = b is
 *   h^d f / prod_l alpha_l: a unit point source f = h^-d at an interior node
 *   is b = 1 there.
 * Memory.  Every array argument is a DEVICE pointer owned by the caller and
 *   borrowed only for the duration of the call (work is enqueued on `stream`
 *   and the call returns after it has completed unless stated otherwise).
 *   The handle owns every internal buffer (factors, workspaces, Krylov basis).
 * Streams.  `stream` is a cudaStream_t (passed as void*); 0 is the legacy
 *   default stream.
 * Errors.  Calls return an hz_status and never throw or abort; hz_last_error
 *   gives a one-line message.  A handle is not thread-safe.
 */
#ifndef HZ_H
#define HZ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } hz_c128;

typedef enum {
  HZ_OK = 0,
  HZ_EINVAL = 1,        /* bad argument (sizes, odd J for the X-sweep, n_rhs > max_rhs, ...) */
  HZ_ENOMEM = 2,        /* device allocation failed */
  HZ_ECUDA = 3,         /* a CUDA call or kernel failed */
  HZ_ENOTFACTORED = 4,  /* hz_solve / hz_precond before hz_factor */
  HZ_ENOTCONV = 5,      /* GMRES hit max_iter; u holds the last iterate, stats are filled */
  HZ_ETIMEOUT = 6,      /* a bounded device-side wait gave up (no hang, context usable) */
  HZ_EINACCURATE = 7    /* a residual norm is not finite (NaN / Inf in the data or operator) */
} hz_status;

/* SweepingPrecUD / SweepingPrecX / SweepingPrecNX (Table 3; NX: partial
 * sweeps inside n_cell groups of subdomains, a comparison pattern) */
enum { HZ_SWEEP_UD = 0, HZ_SWEEP_X = 1, HZ_SWEEP_NX = 2 };
enum { HZ_PLAIN_FP64 = 0, HZ_MIXED = 1 };        /* preconditioner in complex128 / complex64 */

typedef struct {
  int    dim;           /* 2 or 3 */
  int    n[3];          /* interior cells along x (the sweep axis), y, z (n[2]: 3-D only;
                         * even when two_grid) */
  int    w_out;         /* outer layer (PML or sponge) cells per side */
  double h;             /* cell size of every axis (0: 1 / n[0]) */
  double omega;         /* angular frequency; k = omega / c, k^2 = omega^2 m */
  double s_pml_out;     /* outer PML strength S_pml (Section 2.1) */
  double s_pml_dd;      /* DD PML strength (Section 6.1: 15/20/25 for w = 3/4/5) */
  int    J;             /* slabs along x (even for HZ_SWEEP_X) */
  int    w_dd;          /* DD PML width in cells (Section 2.1: 3..5) */
  int    sweep;         /* HZ_SWEEP_UD | HZ_SWEEP_X | HZ_SWEEP_NX */
  int    two_grid;      /* 0: sweep on the fine grid; 1: TGSP (Section 4) */
  int    nu;            /* omega-Jacobi pre- and post-smoothing steps */
  double omega_jac;     /* Jacobi relaxation weight */
  int    precision;     /* HZ_PLAIN_FP64 | HZ_MIXED */
  int    gmres_m;       /* GMRES restart length */
  int    max_iter;      /* cap on preconditioned GMRES iterations */
  double tol;           /* stop at ||b - A u||_2 / ||b||_2 <= tol (per right-hand side) */
  int    max_rhs;       /* right-hand sides per hz_solve call (buffer capacity, 1..64) */
  int    segments;      /* block-row segments per slab solve, over both elimination
                         * chains (0: automatic, about 2 N_y^(2/3) capped at the SM
                         * count; at least 2) */
  double c_pml;         /* PML "typical velocity" (Section 2.1); 0: mean of c over the
                         * unknowns, recomputed by hz_setup / hz_set_medium */
  int    n_cell;        /* HZ_SWEEP_NX: cells N_cell (1..(J+1)/2; cell boundaries
                         * j_cell = 0, round(m (J+1) / N_cell), J+1; centres
                         * j_mid = (j_cell[m-1] + j_cell[m] + 1) / 2); N_cell = 1
                         * is the X-sweep.  Ignored by the other patterns */
  int    boundary;      /* outer layers of w_out cells: HZ_BOUNDARY_PML (Eq. 5) or
                         * HZ_BOUNDARY_SPONGE (Section 2.1: k -> k (1 + i beta), no
                         * PML; beta = sum over the axes of beta_max (d / (w_out h))^2,
                         * d the distance beyond the interior box; two_grid then
                         * coarsens every cell: n[l] + 2 w_out even, Section 4.1) */
  double sponge_damping;/* sponge: one-way amplitude damping exp(-k beta_max w_out h / 3)
                         * of the layer at k = omega / c_pml, in (0, 1) */
  int    block_3d;      /* 3-D slab factorisation: outer block width of the two-level
                         * blocked Gauss-Jordan inverse (the rank of its delayed update,
                         * on the tensor cores in complex64): 64, 128 or 256 (0: 128).
                         * A tuning parameter; the result does not depend on it beyond
                         * rounding */
} hz_params;

enum { HZ_BOUNDARY_PML = 0, HZ_BOUNDARY_SPONGE = 1 };

typedef struct {
  int    n_rhs;
  int    iters_max;        /* max over right-hand sides of GMRES iterations */
  double relres_max;       /* max over right-hand sides of the final true relative residual */
  double t_setup_s;        /* wall time of the last hz_setup / hz_set_medium */
  double t_factor_s;       /* wall time of the last hz_factor */
  double t_solve_s;        /* wall time of the last hz_solve */
  long long precond_applies; /* preconditioner applications in the last hz_solve */
  long long kernel_launches; /* kernels this handle has launched since hz_setup (cumulative) */
} hz_stats;

typedef struct hz_handle hz_handle;

/* Create a solver for the grid and parameters in *p.  m_dev: squared slowness
 * 1/c^2 at the n_dof unknowns, FP64, device, copied into the handle.  c_pml
 * (the "typical velocity" of Section 2.1) is p->c_pml, or the mean of c over
 * the unknowns when p->c_pml is 0.
 * Builds the PML tables (Eq. 5, alpha below Eq. 40), the slab partition
 * (Eq. 17) and the slab meshes (Eqs. 9-10).  *out is NULL on failure. */
hz_status hz_setup(const hz_params* p, const double* m_dev, hz_handle** out);

/* Replace the medium (same grid); invalidates the factors. */
hz_status hz_set_medium(hz_handle* h, const double* m_dev);

/* Factor every slab operator A^(j) (Section 2.2; Section 5: the paper uses a
 * sparse direct solver here): a twisted block LU along y whose two
 * elimination chains start at the outer PML rows and meet in the middle row,
 * plus the segment transfer products of the parallel-in-y slab solve. */
hz_status hz_factor(hz_handle* h, void* stream);

/* Solve A u_r = f_r for r < n_rhs by GMRES(m) with the configured
 * preconditioner, x0 = 0.  f_dev, u_dev: n_rhs * n_dof complex128, device.
 * stats (host, may be NULL) is filled.  Returns HZ_ENOTCONV if any right-hand
 * side missed tol within max_iter (u holds the last iterate). */
hz_status hz_solve(hz_handle* h, const hz_c128* f_dev, hz_c128* u_dev, int n_rhs,
                   void* stream, hz_stats* stats);

/* Same as hz_solve with HOST arrays f_host / u_host (n_rhs * n_dof complex128,
 * pinned or pageable): the host<->device copies are part of the call.  The
 * first call allocates two device staging buffers owned by the handle. */
hz_status hz_solve_host(hz_handle* h, const hz_c128* f_host, hz_c128* u_host, int n_rhs,
                        void* stream, hz_stats* stats);

/* Components of the path, exposed for testing and composition. */

/* y = A u (Eq. 40 x h^d), complex128, n_rhs fields. */
hz_status hz_apply(hz_handle* h, const hz_c128* u_dev, hz_c128* y_dev, int n_rhs, void* stream);

/* z = M r: one application of the configured preconditioner (SweepingPrecX /
 * SweepingPrecUD of Table 3, or the TGSP of Section 4), complex128 in and out
 * (computed in the preconditioner precision). */
hz_status hz_precond(hz_handle* h, const hz_c128* r_dev, hz_c128* z_dev, int n_rhs, void* stream);

/* Receiver misfit and its gradient with respect to the squared slowness m
 * (the adjoint-state method; the paper supplies the solver, Eq. 40 the
 * derivative of A):
 *   Phi = 1/2 sum_s sum_q |u_s[rec_q] - d[s][q]|^2,  A u_s = e_{src_s} (b = 1),
 *   grad[i] = dPhi/dm_i = omega^2 Re( h^d / (prod_l alpha_l)_i sum_s mu_{s,i} u_{s,i} ),
 * with A mu_s = conj(sum_q (u_s[rec_q] - d[s][q]) e_{rec_q}) (A is complex
 * symmetric, so the adjoint solve reuses the preconditioner) and the PML held
 * fixed (set p->c_pml to keep it fixed across hz_set_medium calls).
 * src_dev: n_src flat unknown indices (int32, device); rec_dev: n_rec flat
 * indices (int32, device; repeats add up); d_dev: observed data [n_src][n_rec]
 * complex128 (device); grad_dev: n_dof doubles (device, overwritten); *phi
 * (host) receives Phi.  Sources are solved max_rhs at a time (one forward and
 * one adjoint GMRES solve per batch).  Indices outside the grid give
 * HZ_EINVAL before any work; HZ_ENOTCONV if a solve missed tol (results are
 * still written).  Requires hz_factor.  The first call allocates
 * 3 * max_rhs * n_dof complex128 of work space owned by the handle. */
hz_status hz_grad(hz_handle* h, const int* src_dev, int n_src, const int* rec_dev,
                         int n_rec, const hz_c128* d_dev, double* grad_dev, double* phi,
                         void* stream, hz_stats* stats);

/* Geometry of slab j (1..J) on the sweep level: global core columns lo..hi,
 * added PML columns wl (left) / wr (right), width W = hi-lo+1+wl+wr. */
hz_status hz_slab_info(const hz_handle* h, int j, int* lo, int* hi, int* wl, int* wr, int* W);

/* Layout of the parallel-in-y slab substitution (the twisted block LU that
 * implements SubdomSolve, Table 2) for a slab of ny block rows; host only, no
 * handle and no GPU needed.  segments: as hz_params.segments (<= 0:
 * automatic, about 2 ny^(2/3), capped at max_auto; hz_setup uses twice the SM
 * count in mixed precision, the SM count in plain FP64).  Outputs (host):
 * *mid = the row where the two elimination chains meet, *P segments, the
 * first *S0 on the top chain, *NG segment groups of the two-level carries,
 * the first *G0 on the top chain.  seg_out (capacity seg_cap entries of 4
 * ints, may be NULL): per segment first row, rows, direction (+1 top chain,
 * -1 bottom chain), group; grp_out (capacity grp_cap entries of 4 ints, may be
 * NULL): per group first segment, last segment, half (0 top, 1 bottom), index
 * within the half.  HZ_EINVAL for ny < 3, a NULL count pointer or a capacity
 * below the counts (the counts are still written). */
hz_status hz_segment_layout(int ny, int segments, int max_auto, int* mid, int* P, int* S0,
                            int* NG, int* G0, int* seg_out, int seg_cap, int* grp_out,
                            int grp_cap);

/* u_d = (A^(j))^-1 f_d for slab j (1..J) of the sweep level: f_dev, u_dev are
 * n_rhs * N_t * W complex128 ([rhs][y][local x]).  Requires hz_factor. */
hz_status hz_slab_solve(hz_handle* h, int j, const hz_c128* f_dev, hz_c128* u_dev, int n_rhs,
                        void* stream);

/* hz_slab_solve without any device allocation.  (The paper has no
 * counterpart.)  It serves callers that must not allocate device memory
 * once they are running: real-time or embedded schedulers that forbid
 * allocation after start-up, and applications that hand all device memory
 * to their own pool allocator, where a cudaMalloc inside the library could
 * fail or fragment that pool.  Same arguments, layout and result as
 * hz_slab_solve.  Its work space is a fixed 8 MiB device array inside the
 * library, present on every GPU that loads the library until the process
 * exits; a call needing more (about 3 * n_rhs * N_t * W complex values in
 * mixed precision, n_rhs * N_t * W in FP64, plus segment carries) returns
 * HZ_EINVAL before any GPU work.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it; do not call this entry point after cudaDeviceReset (the kept
 * address would be stale).  All calls share the one array and it keeps the last call's
 * contents: calls whose GPU work overlaps (two streams, two host threads)
 * race and give wrong results.  The call synchronises `stream` before
 * returning.  Requires hz_factor. */
hz_status hz_slab_solve_noalloc(hz_handle* h, int j, const hz_c128* f_dev, hz_c128* u_dev,
                                int n_rhs, void* stream);

/* Statistics of the last call; fills *out. */
hz_status hz_get_stats(const hz_handle* h, hz_stats* out);

/* Kernel-level timing for roofline reporting.  hz_enable_timing(h, 1) resets
 * the counters and brackets every launch of a tagged kernel with two CUDA
 * events on the stream it is launched on (0 disables).  hz_kernel_timing
 * returns, for one tag, the summed event time (ms), the number of launches
 * and the algorithmic bytes those launches move (method minimum: each
 * factor block read once per pass, vectors once).  Tags: "slab_solve" (one
 * whole subdomain solve of SubdomSolve, Table 2), its kernels "slab_rhs",
 * "slab_fwd_pass1", "slab_carry" (in-group segment carries),
 * "slab_carry_bound" (group boundary carries), "slab_fwd_bwd1", "slab_bwd";
 * the factorisation kernels "slab_factor" (on devices with cooperative
 * launch: the elimination chains together with the operator, segment and
 * prefix products), "slab_middle", and, without cooperative launch,
 * "segment_product" and "segment_prefix" (bytes 0); the matrix-free operator
 * "stencil_c64", "stencil_c128" (Eq. 40 apply, residual, Jacobi step).
 * Unknown tags return zeros. */
hz_status hz_enable_timing(hz_handle* h, int on);
hz_status hz_kernel_timing(hz_handle* h, const char* tag, double* ms, long long* launches,
                           double* bytes);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (2 flop per FMA), FP32 for precision = HZ_MIXED, FP64 for HZ_PLAIN_FP64:
 * the denominator of the ALU rooflines of the factorisation kernels.  (The
 * paper has no counterpart: a measurement utility.)  Runs about a second of
 * FMA chains on every SM of the device on `stream`; *tflops (host) receives
 * the best of three timed launches.  HZ_EINVAL for a NULL pointer or another
 * precision value. */
hz_status hz_alu_peak(int precision, double* tflops, void* stream);

/* Test hooks (environment variables, read at every call; unset in
 * production).  HZ_TEST_ALLOC_LIMIT=<bytes>: every device allocation of at
 * least that size fails as an out-of-memory error (HZ_ENOMEM paths).
 * HZ_TEST_WAIT_LIMIT_NS=<ns>: limit of the fused factorisation's bounded
 * wait for elimination-chain progress (default 10 s); 0 makes the waiting
 * CTAs give up at once, so hz_factor returns HZ_ETIMEOUT without any hang.
 * HZ_TEST_NO_COOP=1: factor with separate launches, as on devices without
 * cooperative launch. */

const char* hz_last_error(const hz_handle* h);
const char* hz_status_string(hz_status s);
void hz_destroy(hz_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
