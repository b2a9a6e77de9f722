"""The C-ABI library builds, loads and exports every symbol of include/hz.h;
argument validation that needs no GPU returns HZ_EINVAL."""

import ctypes

import pytest

import paper_1412_0464_gb300 as hz


@pytest.fixture(scope="module")
def L():
    hz.build()
    return hz.lib()


def test_exports_every_declared_symbol(L):
    names = hz.declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hz._SIGNATURES)


def _params(**kw):
    p = hz.hz_params()
    base = dict(dim=2, n=40, w_out=5, omega=50.0, s_pml_out=20.0, s_pml_dd=20.0, J=4, w_dd=4,
                sweep=hz.HZ_SWEEP_X, two_grid=0, nu=3, omega_jac=0.8, precision=hz.HZ_PLAIN_FP64,
                gmres_m=20, max_iter=100, tol=1e-6, max_rhs=1, segments=0)
    base.update(kw)
    for k, v in base.items():
        if k == "n":                       # interior cells along x, y, z
            for l, c in enumerate(v if isinstance(v, tuple) else (v, v, v)):
                p.n[l] = c
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [dict(dim=4), dict(dim=1), dict(J=3), dict(n=2),
                                 dict(n=(40, 2, 40)), dict(dim=3, n=(40, 40, 3)), dict(max_rhs=0),
                                 dict(max_rhs=99), dict(tol=0.0), dict(w_dd=0), dict(J=60),
                                 dict(precision=7), dict(sweep=5), dict(h=-1.0),
                                 dict(two_grid=1, n=(40, 41, 40)), dict(boundary=2),
                                 dict(boundary=1, sponge_damping=0.0),
                                 dict(boundary=1, sponge_damping=1.5),
                                 dict(boundary=1, sponge_damping=0.01, w_out=0),
                                 dict(sweep=hz.HZ_SWEEP_NX, n_cell=0),
                                 dict(sweep=hz.HZ_SWEEP_NX, n_cell=3), dict(block_3d=96),
                                 dict(block_3d=-1)])
def test_setup_rejects_bad_parameters(L, bad):
    h = ctypes.c_void_p()
    st = L.hz_setup(ctypes.byref(_params(**bad)), ctypes.c_void_p(1), ctypes.byref(h))
    assert st == hz.HZ_EINVAL
    assert h.value is None
    assert L.hz_last_error(None)


def test_null_handle_calls(L):
    assert L.hz_factor(None, None) == hz.HZ_EINVAL
    assert L.hz_solve(None, None, None, 1, None, None) == hz.HZ_EINVAL
    assert L.hz_status_string(hz.HZ_ENOTCONV) == b"HZ_ENOTCONV"
    L.hz_destroy(None)
