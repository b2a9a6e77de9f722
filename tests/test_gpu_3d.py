"""3-D path, rectangular grids and many right-hand sides: parity with the FP64 oracle.

3-D: the 7-point fine operator (Eq. 40 in 3-D), the 27-point coarse FE
operator (Appendix A, Eq. 63, Table 9(b)), the dense-block twisted LU of the
3-D slabs (block rows = z layers of N_y W unknowns), the 3-D transmission
planes (Eqs. 19-20), SweepingPrecX / UD (Table 3), the two-grid cycle
(Section 4) and GMRES, on reduced versions of the 3-D workloads (layered
medium of configuration 4, random medium and two-grid of configuration 5)
with ragged slab widths.  The oracle is dimension-generic (and pinned in 3-D).

Tolerances as in the 2-D parity tests: FP64 operators 1e-12, FP64 slab solves
and preconditioners 1e-9; complex64 (mixed) slab solves and preconditioners
3e-4 (relative L2 and element-wise against the largest entry); GMRES
solutions 1e-5 against the oracle's direct solve with relative residual
<= 1e-6.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import adjoint
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-9, "mixed": 3e-4}


def _hz():
    import paper_1412_0464_gb300 as hz
    hz.build()
    return hz


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _close(a, b, tol):
    return _rel(a, b) <= tol and np.abs(a - b).max() <= tol * np.abs(b).max()


# (config, n, w_out, J): 3-D finite differences (config 4 recipe) and two-grid (config 5)
FD3 = [(4, 16, 4, 4), (4, 18, 3, 2)]
TG3 = [(5, 24, 4, 2), (5, 32, 4, 4)]


@pytest.mark.parametrize("idx,n,w_out,J", FD3)
def test_apply_3d_matches_oracle(idx, n, w_out, J):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=2)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision="fp64")
    u = _rand((2,) + cfg.shape, 1)
    y = s.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    for r in range(2):
        ref = (p.A @ u[r].ravel()).reshape(cfg.shape)
        assert np.abs(y[r] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J", FD3 + TG3)
def test_slab_solve_3d_matches_oracle(idx, n, w_out, J, precision):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=3)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision=precision)
    s.factor()
    for j in range(1, J + 1):
        sl = p.dd.slabs[j]
        info = s.slab_info(j)
        assert (info["lo"], info["hi"], info["wl"], info["wr"], info["W"]) == \
            (sl.lo, sl.hi, sl.wl, sl.wr, sl.W)
        nt = sl.A.shape[0] // sl.W
        fd = _rand((3, nt, sl.W), 10 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        for r in range(3):
            ref = sl.lu.solve(fd[r].ravel()).reshape(nt, sl.W)
            assert _close(ud[r], ref, TOL[precision]), (j, r, _rel(ud[r], ref))


@pytest.mark.parametrize("sweep", ["X", "UD"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J", [FD3[0], TG3[0]])
def test_preconditioner_3d_matches_oracle(idx, n, w_out, J, precision, sweep):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=2)
    p = Problem(cfg, sweep=sweep)
    s = hz.Solver.from_workload(cfg, precision=precision, sweep=sweep)
    s.factor()
    f = _rand((2,) + cfg.shape, 3)
    z = s.precond(torch.from_numpy(f).cuda()).cpu().numpy()
    for r in range(2):
        ref = p.precondition(f[r]).reshape(cfg.shape)
        assert _close(z[r], ref, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx,n,w_out,J", [FD3[0], TG3[0]])
def test_solve_3d_matches_direct_solve(idx, n, w_out, J, precision):
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=3)
    p = Problem(cfg)
    b = synth.sources(cfg)
    s = hz.Solver.from_workload(cfg, precision=precision)
    s.factor()
    u, st = s.solve(torch.from_numpy(b).cuda())
    u = u.cpu().numpy()
    lu = spla.splu(p.A.tocsc())
    for r in range(3):
        exact = lu.solve(b[r].ravel()).reshape(cfg.shape)
        relres = np.linalg.norm(p.A @ u[r].ravel() - b[r].ravel()) / np.linalg.norm(b[r])
        assert relres <= 1.05 * cfg.tol
        assert _rel(u[r], exact) <= 1e-5
    assert st["relres_max"] <= cfg.tol
    if precision == "fp64":
        _, info = p.solve(b[0])
        assert abs(st["iters_max"] - info["iters"]) <= 1


@pytest.mark.parametrize("dims,two_grid", [((48, 64), False), ((40, 56), True), ((72, 40), False)])
def test_rectangle_2d(dims, two_grid):
    """2-D rectangles (n_y != n_x): operator, preconditioner and solve."""
    hz = _hz()
    cfg = synth.scaled_workload(3 if two_grid else 2, dims[-1], w_out=6, J=4, dims=dims)
    assert cfg.shape[0] != cfg.shape[1]
    p = Problem(cfg)
    for precision in ("fp64", "mixed"):
        s = hz.Solver.from_workload(cfg, precision=precision, max_rhs=2)
        s.factor()
        u = _rand((2,) + cfg.shape, 4)
        if precision == "fp64":
            y = s.apply(torch.from_numpy(u).cuda()).cpu().numpy()
            ref = (p.A @ u[0].ravel()).reshape(cfg.shape)
            assert np.abs(y[0] - ref).max() <= 1e-12 * np.abs(ref).max()
        z = s.precond(torch.from_numpy(u).cuda()).cpu().numpy()
        assert _close(z[1], p.precondition(u[1]).reshape(cfg.shape), TOL[precision])
        b = synth.sources(cfg)[0]
        x, st = s.solve(torch.from_numpy(b).cuda())
        exact = spla.spsolve(p.A.tocsc(), b.ravel()).reshape(cfg.shape)
        assert _rel(x.cpu().numpy(), exact) <= 1e-5 and st["relres_max"] <= cfg.tol
        s.close()


@pytest.mark.parametrize("idx,n,w_out,J,nr", [(2, 60, 6, 4, 12), (4, 14, 3, 2, 10)])
def test_many_right_hand_sides(idx, n, w_out, J, nr):
    """More than 8 right-hand sides per call (the slab solves take them in chunks of 8)."""
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision="mixed", max_rhs=nr)
    s.factor()
    f = _rand((nr,) + cfg.shape, 6)
    z = s.precond(torch.from_numpy(f).cuda()).cpu().numpy()
    for r in (0, 7, 8, nr - 1):
        assert _close(z[r], p.precondition(f[r]).reshape(cfg.shape), TOL["mixed"])
    b = _rand((nr,) + cfg.shape, 7)
    u, st = s.solve(torch.from_numpy(b).cuda())
    u = u.cpu().numpy()
    lu = spla.splu(p.A.tocsc())
    for r in range(nr):
        assert _rel(u[r], lu.solve(b[r].ravel()).reshape(cfg.shape)) <= 1e-5
    assert st["n_rhs"] == nr and st["relres_max"] <= cfg.tol


def test_gradient_3d_matches_oracle():
    """hz_grad in 3-D (two-grid, mixed) against the oracle adjoint (exact solves)."""
    hz = _hz()
    cfg = synth.scaled_workload(5, 16, w_out=4, J=2, n_src=3, n_rec=4)
    m_true, m0 = synth.medium(cfg, "true"), synth.medium(cfg, "start")
    c_pml = float(np.mean(1.0 / np.sqrt(m0)))
    src = np.array([np.ravel_multi_index(tuple(int(v) for v in idx), cfg.shape)
                    for idx in synth.source_nodes(cfg)])
    rec = synth.receivers(cfg)
    d = adjoint.synthetic_data(Problem(cfg, m_true, two_grid=False, c_pml=c_pml), src, rec)
    s = hz.Solver.from_workload(cfg, m=m0, tol=1e-10, c_pml=c_pml, max_rhs=2)
    s.factor()
    phi, g, st = s.grad(src, rec, d)
    phi_o, g_o, _ = adjoint.misfit_and_gradient(Problem(cfg, m0, two_grid=False, c_pml=c_pml),
                                                src, rec, d)
    g = g.cpu().numpy()
    assert phi > 0 and abs(phi - phi_o) <= 1e-8 * phi_o
    assert np.abs(g - g_o).max() <= 1e-7 * np.abs(g_o).max()


@pytest.mark.parametrize("idx,n,w_out,J", [(4, 24, 4, 2), (5, 40, 4, 2)])
def test_tensor_core_update_matches_simt_and_oracle(idx, n, w_out, J, monkeypatch):
    """The complex64 3-D factorisation updates S outside each outer block of
    128 columns on the tensor cores (three TF32 passes per real product), and
    slab solves with 8 right-hand sides multiply by the stored inverses on the
    tensor cores too.  Blocks of B = 31 x 19 = 589 (finite differences) and
    27 x 17 = 459 (two-grid coarse level) unknowns span several outer blocks
    and a ragged last one; the slab solves agree with the FP32 SIMT kernels
    (HZ_TEST_NO_TC=1) and with the oracle's exact slab solves."""
    hz = _hz()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=8)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision="mixed")
    fds = {}
    for j in range(1, J + 1):
        sl = p.dd.slabs[j]
        nt = sl.A.shape[0] // sl.W
        fds[j] = _rand((8, nt, sl.W), 40 + j)
    out = {}
    for mode in ("tc", "simt"):
        if mode == "simt":
            monkeypatch.setenv("HZ_TEST_NO_TC", "1")
        s.factor()
        out[mode] = {j: s.slab_solve(j, torch.from_numpy(fds[j]).cuda()).cpu().numpy()
                     for j in fds}
    for j, fd in fds.items():
        sl = p.dd.slabs[j]
        nt = sl.A.shape[0] // sl.W
        for r in range(8):
            ref = sl.lu.solve(fd[r].ravel()).reshape(nt, sl.W)
            assert _close(out["tc"][j][r], ref, TOL["mixed"]), (j, r, _rel(out["tc"][j][r], ref))
            assert _close(out["tc"][j][r], out["simt"][j][r], TOL["mixed"])


def test_slab_solve_3d_40_rhs_two_tensor_core_chunks():
    """40 right-hand sides: the tensor-core layer products run in two chunks
    of 32 (the second one partly filled) and one reduction; every solution
    matches the oracle's exact slab solve."""
    hz = _hz()
    cfg = synth.scaled_workload(4, 16, w_out=4, J=2, n_src=40)
    p = Problem(cfg)
    s = hz.Solver.from_workload(cfg, precision="mixed")
    s.factor()
    for j in (1, 2):
        sl = p.dd.slabs[j]
        nt = sl.A.shape[0] // sl.W
        fd = _rand((40, nt, sl.W), 70 + j)
        ud = s.slab_solve(j, torch.from_numpy(fd).cuda()).cpu().numpy()
        for r in (0, 17, 31, 32, 39):
            ref = sl.lu.solve(fd[r].ravel()).reshape(nt, sl.W)
            assert _close(ud[r], ref, TOL["mixed"]), (j, r, _rel(ud[r], ref))


@pytest.mark.gpu
@pytest.mark.parametrize("n", [36, 44])
def test_slab_solve_3d_blocks_beyond_1024_rows_mixed_matches_fp64(n):
    """Dense blocks of more than 1024 unknowns: 43 x 25 and 43 x 26 (n = 36),
    51 x 29 and 51 x 30 (n = 44).  The complex64 panels hold three rows per
    thread in registers up to 1344 rows, and beyond that two, with rows 1024
    and up in shared memory.  The complex128 blocks are too large for the
    shared-memory panel and take the global-memory one.  8 right-hand sides run
    the tensor-core layer products, with the packed right-hand sides formed by
    the coupling kernel and by the reductions.  At this size the oracle's
    sparse LU of a slab takes too long, so the mixed solve is checked against
    the FP64 solve (itself matched to the oracle at the sizes above) within
    the complex64 tolerance."""
    hz = _hz()
    cfg = synth.scaled_workload(4, n, w_out=4, J=2, n_src=8)
    s64 = hz.Solver.from_workload(cfg, precision="fp64")
    s64.factor()
    s32 = hz.Solver.from_workload(cfg, precision="mixed")
    s32.factor()
    nt = cfg.shape[1] * cfg.shape[2]
    for j in (1, 2):
        W = s32.slab_info(j)["W"]
        assert cfg.shape[1] * W > 1024
        fd = torch.from_numpy(_rand((8, nt, W), 90 + j)).cuda()
        u64 = s64.slab_solve(j, fd).cpu().numpy()
        u32 = s32.slab_solve(j, fd).cpu().numpy()
        for r in range(8):
            assert _close(u32[r], u64[r], TOL["mixed"]), (j, r, _rel(u32[r], u64[r]))
