"""The C-ABI library loads, exports every declared entry point and validates
its arguments on the host (no GPU needed; no compute calls are made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:cpd_status|const char\s*\*)\s*(cpd_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def cpd():
    from paper_2103_04081_gb300 import build
    build.build()
    from paper_2103_04081_gb300 import cpd as C
    return C


def test_exports_every_declared_symbol(cpd):
    names = declared_symbols()
    assert {"cpd_init", "cpd_sgd_iters", "cpd_fit", "cpd_destroy"} <= names
    for name in sorted(names):
        assert hasattr(cpd.lib(), name), name


def _init_status(cpd, **kw):
    import torch
    cfg = cpd.make_config(**kw)
    X = torch.zeros(8)
    A0 = [torch.zeros(2, 1) for _ in kw["dims"]]
    ctx = ctypes.c_void_p()
    st = cpd.lib().cpd_init(ctypes.byref(cfg), X.data_ptr(), cpd.HOST,
                            (ctypes.c_void_p * len(A0))(*[a.data_ptr() for a in A0]),
                            cpd.HOST, None, ctypes.byref(ctx))
    return st, cpd.lib().cpd_last_error().decode()


@pytest.mark.parametrize("kw,msg", [
    (dict(dims=(2, 2), R=1, B=1), "N must"),
    (dict(dims=(2, 2, 2), R=0, B=1), "R must"),
    (dict(dims=(2, 2, 2), R=1, B=0), "B must"),
    (dict(dims=(3, 3, 3), R=3, B=1, sampling="leverage"), "I_k > R"),
    (dict(dims=(2, 2, 2), R=1, B=1, step="adagrad", eta=0.0), "eta"),
    (dict(dims=(2, 2, 2), R=1, B=1, step="decay", gamma=0.0), "gamma"),
    (dict(dims=(2, 2, 2), R=1, B=1, x_dtype="f32", engine="tensor"), "tensor-core"),
    (dict(dims=(8, 8, 8), R=1, B=4, tile_rows=12), "tile_rows must be a multiple of 8"),
    (dict(dims=(8, 8, 8), R=1, B=4, tile_fibers=5), "tile_fibers <= B"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="tensor", tile_fibers=20), "tensor-core engines"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="tensor", tile_rows=64), "tensor-core engines"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="persistent", tile_fibers=32), "take no tile_rows"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="fused", tile_fibers=32), "take no tile_rows"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="fused", max_ctas=3), "cluster size"),
    (dict(dims=(64, 64, 64), R=16, B=4000, engine="fused", max_ctas=16), "208 fibers"),
    (dict(dims=(64, 64, 64), R=16, B=64, x_dtype="f32", engine="fused"), "tensor-core engine"),
    (dict(dims=(8, 8, 8), R=1, B=4, block=3), "must divide B, I_1 and I_2"),
    (dict(dims=(6, 8, 8), R=1, B=8, block=4), "must divide B, I_1 and I_2"),
    (dict(dims=(8, 8, 8), R=1, B=8, block=-1), "block must be >= 0"),
    (dict(dims=(64, 64, 64), R=16, B=64, block=2, engine="persistent"), "samples fibers one by one"),
    (dict(dims=(8, 8, 8), R=1, B=4, x_layout="strided", engine="cluster"), "strided x_layout"),
    (dict(dims=(0, 2, 2), R=1, B=1), "every dim must be in [1, 2^31]"),
    (dict(dims=(2, 2**31 + 1, 2), R=1, B=1), "every dim must be in [1, 2^31]"),
    (dict(dims=(2**20, 2**20, 2**20), R=1, B=1), "tensor too large"),
    (dict(dims=(2, 2, 2), R=1, B=1, step="adagrad", eta=0.1, b=-1.0), "AdaGrad needs eta > 0 and b >= 0"),
    (dict(dims=(8, 8, 8), R=1, B=4, tile_rows=520), "tile_rows must be a multiple of 8"),
    (dict(dims=(64, 64, 64), R=16, B=512, engine="cluster", tile_fibers=272), "tensor-core engines"),
    (dict(dims=(64, 64, 64), R=16, B=512, engine="tensor", tile_fibers=144), "tensor-core engines"),
    (dict(dims=(64, 64, 64), R=80, B=64, engine="cluster"), "R <= 64"),
    (dict(dims=(1100, 64, 64), R=16, B=64, engine="cluster"), "every I_k <= 1024"),
    (dict(dims=(64, 64, 64), R=16, B=64, engine="persistent", max_ctas=32), "at most 16"),
    (dict(dims=(64, 64, 64), R=16, B=64, x_dtype="f32", engine="persistent"), "persistent engine needs BF16"),
    (dict(dims=(64, 64, 64), R=16, B=64, sampling="leverage", engine="persistent"), "persistent engine needs BF16"),
])
def test_invalid_configs_rejected_on_host(cpd, kw, msg):
    st, err = _init_status(cpd, **kw)
    assert st == cpd.EINVAL
    assert msg in err


def test_unknown_constraint_and_layout_rejected(cpd):
    import torch
    for field, value, msg in (("constraint", 7, "constraint"), ("x_layout", 2, "x_layout"),
                              ("max_ctas", -1, "max_ctas"), ("N", 9, "N must"), ("R", 257, "R must"),
                              ("B", 65537, "B must"), ("sampling", 3, "unknown sampling"),
                              ("step", 3, "unknown step"), ("x_dtype", 3, "unknown x_dtype"),
                              ("engine", 6, "unknown engine"), ("engine", -1, "unknown engine")):
        cfg = cpd.make_config(dims=(2, 2, 2), R=1, B=1)
        setattr(cfg, field, value)
        X = torch.zeros(8)
        A0 = [torch.zeros(2, 1) for _ in range(3)]
        ctx = ctypes.c_void_p()
        st = cpd.lib().cpd_init(ctypes.byref(cfg), X.data_ptr(), cpd.HOST,
                                (ctypes.c_void_p * 3)(*[a.data_ptr() for a in A0]),
                                cpd.HOST, None, ctypes.byref(ctx))
        assert st == cpd.EINVAL
        assert msg in cpd.lib().cpd_last_error().decode()


def test_no_cpu_fallback(cpd):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, err = _init_status(cpd, dims=(2, 2, 2), R=1, B=1)
    assert st == cpd.ECUDA, err


def test_server_group_and_variance_reject_bad_arguments_on_host(cpd):
    """Argument checks that come before any device work."""
    import ctypes as C
    cfg = cpd.cpd_server_config()
    cfg.strided_above_mb = -1
    srv = C.c_void_p()
    assert cpd.lib().cpd_server_create(C.byref(cfg), C.byref(srv)) == cpd.EINVAL
    cfg = cpd.cpd_server_config()
    cfg.no_grouping = 2
    assert cpd.lib().cpd_server_create(C.byref(cfg), C.byref(srv)) == cpd.EINVAL
    grp = C.c_void_p()
    assert cpd.lib().cpd_group_create(None, 1, None, C.byref(grp)) == cpd.EINVAL
    arr = (C.c_void_p * 1)(None)
    assert cpd.lib().cpd_group_create(arr, 0, None, C.byref(grp)) == cpd.EINVAL
    assert cpd.lib().cpd_group_create(arr, 1, None, C.byref(grp)) == cpd.EINVAL
    assert cpd.lib().cpd_group_iters(None, 1, None) == cpd.EINVAL
    assert cpd.lib().cpd_group_destroy(None) == cpd.OK
    v = C.c_double()
    assert cpd.lib().cpd_grad_variance(None, 0, C.byref(v), None, None) == cpd.EINVAL
    assert cpd.lib().cpd_server_destroy(None) == cpd.OK


def _header_arity():
    """Parameter count of every cpd_status function declared in include/*.h."""
    arity = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
        for m in re.finditer(r"cpd_status\s+(cpd_\w+)\s*\(([^)]*)\)\s*;", txt):
            params = m.group(2).strip()
            arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_signatures_match_the_header(cpd):
    """The ctypes argument lists of the binding have the header's arity, so no
    call passes a shifted argument."""
    arity = _header_arity()
    assert len(arity) >= 30, sorted(arity)
    for name, n in sorted(arity.items()):
        f = getattr(cpd.lib(), name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)


def test_null_handles_rejected_on_host(cpd):
    """Every call on a context, group or server rejects a NULL handle with
    CPD_EINVAL before any device work; the destroy calls accept NULL."""
    L = cpd.lib()
    calls = {
        "cpd_sgd_iters": (None, 1, None), "cpd_prepare": (None, 1, None),
        "cpd_gradients": (None, 0, 0, 1, None, None), "cpd_skrp": (None, 0, 0, 1, None, None, None, None, None),
        "cpd_fit": (None, None, None, None), "cpd_fit_start": (None, None), "cpd_fit_poll": (None, None, None),
        "cpd_get_factors": (None, None, 0, None), "cpd_set_factors": (None, None, 0, None),
        "cpd_get_adagrad": (None, None, 0, None), "cpd_set_adagrad": (None, None, 0, None),
        "cpd_get_iteration": (None, None), "cpd_set_iteration": (None, 0),
        "cpd_last_sample": (None, None, None, None, None), "cpd_last_gradient": (None, None, None),
        "cpd_sync": (None, None), "cpd_profile": (None, 1), "cpd_profile_read": (None, None, None, None, None),
        "cpd_trace": (None, 1), "cpd_trace_read": (None, None, None), "cpd_describe": (None, None, 0),
        "cpd_grad_variance": (None, 0, None, None, None), "cpd_group_create": (None, 1, None, None),
        "cpd_group_iters": (None, 1, None), "cpd_submit": (None, None, None, 0, None, 0, 0.0, 1, None),
        "cpd_poll": (None, 0, None, None), "cpd_server_wait": (None, 1.0),
        "cpd_server_stats": (None, None, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == cpd.EINVAL, name
    for name in ("cpd_destroy", "cpd_group_destroy", "cpd_server_destroy"):
        assert getattr(L, name)(None) == cpd.OK, name
