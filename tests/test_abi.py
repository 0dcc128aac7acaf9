"""The C-ABI library builds, loads and exports every entry point include/dbar.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dbar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dbar_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_02363_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dbar_plan_create", "dbar_plan_destroy", "dbar_solve_cgo", "dbar_apply", "dbar_rhs",
                     "dbar_m_from_S", "dbar_taylor", "dbar_fft2", "dbar_last_error", "dbar_params_init"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol(lib):
    from paper_1508_02363_gb300 import dbar
    for name in declared_functions():
        assert hasattr(dbar, name), name


def test_parameter_validation_is_host_side(lib):
    from paper_1508_02363_gb300 import dbar
    for bad in (dict(N=48), dict(N=16), dict(N=4096), dict(L=0.0), dict(M=17), dict(restart=0),
                dict(tol=0.0), dict(prec=7), dict(sstep=3), dict(sstep=8), dict(sstep=4, restart=30),
                dict(iterated=2), dict(regularisation=2),
                dict(regularisation=1), dict(regularisation=1, prec=0, N=512),
                dict(regularisation=1, prec=0, iterated=1),
                dict(regularisation=1, prec=0, max_batch=5000), dict(inner_M=3), dict(inner_M=-1), dict(autotune=4),
                dict(gauss_w=0.0), dict(gauss_w=-1.0), dict(gauss_w=float("nan")), dict(support_skip=2), dict(row_shape=6), dict(row_shape=-1),
                dict(row_shape_plain=6), dict(row_shape_plain=-1)):
        args = dict(N=64, L=4.0)
        args.update(bad)
        p = dbar.dbar_params_init(args.pop("N"), args.pop("L"), **args)
        with pytest.raises(dbar.DbarError) as e:
            dbar.dbar_plan_create(p)
        assert e.value.status == dbar.DBAR_EINVAL, bad
    with pytest.raises(dbar.DbarError):
        dbar.dbar_solve_cgo(None, None, [0.1], None)


def test_params_defaults_and_solve_signature(lib):
    # the struct as the header lays it out, filled by the library's own defaults
    from paper_1508_02363_gb300 import dbar
    p = dbar.dbar_params_init(128, 5.0)
    assert (p.N, p.L, p.M, p.restart, p.gauss_w, p.mem_budget, p.support_skip) == (128, 5.0, 2, 32, 1.0, 0, 1)
    # dbar_solve_cgo(plan, Q, nk, k, x0, S_out, m_out, iters, resid, io_on_device, stream):
    # eleven arguments, a NULL plan answered on the host
    assert len(lib.dbar_solve_cgo.argtypes or dbar._lib.dbar_solve_cgo.argtypes) == 11
    k = (ctypes.c_double * 2)(0.1, 0.0)
    st = dbar._lib.dbar_solve_cgo(None, None, 1, k, None, None, None, None, None, 0, None)
    assert st == dbar.DBAR_EINVAL and "plan" in dbar.dbar_last_error()


def test_row_tuning_rejects_a_null_plan(lib):
    from paper_1508_02363_gb300 import dbar
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_plan_row_tuning(None, "plain")
    assert e.value.status == dbar.DBAR_EINVAL
    with pytest.raises(ValueError):
        dbar.dbar_plan_row_tuning(None, "columns")


def test_wait_hook_rejects_a_null_plan(lib):
    from paper_1508_02363_gb300 import dbar
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_plan_inject_wait_timeout(None)
    assert e.value.status == dbar.DBAR_EINVAL


def test_batches_reject_a_missing_plan(lib):
    from paper_1508_02363_gb300 import dbar
    import numpy as np
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_solve_batches([{"plan": None, "Q": np.zeros((32, 32), complex), "k": [0.1],
                                  "S_out": np.zeros((1, 32, 32), complex)}], stream=0)
    assert e.value.status == dbar.DBAR_EINVAL
