"""Host-only checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point that include/gt_avalanche.h
declares, its struct layouts match the binding, and calls that need no
device behave as documented."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2509_15377_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gt_avalanche.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2509_15377_gb300 import build as B
    B.build()
    from paper_2509_15377_gb300 import avalanche as A
    return A.load()


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("sizeof",)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2509_15377_gb300 import avalanche as A
    names = declared_functions()
    assert set(names) == set(A.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match(lib):
    from paper_2509_15377_gb300 import avalanche as A
    sizes = (C.c_size_t * 5)()
    assert lib.gt_abi_sizes(sizes, 5) == 0
    assert list(sizes) == [C.sizeof(s) for s in (A.gt_gas, A.gt_field, A.gt_run,
                                                    A.gt_endpoints, A.gt_stats)]
    assert lib.gt_abi_sizes(sizes, 4) == A.GT_ERR_ARG
    assert lib.gt_abi_version() == A.GT_ABI_VERSION == 4


def test_error_strings(lib):
    from paper_2509_15377_gb300 import avalanche as A
    for code in (A.GT_OK, A.GT_ERR_ARG, A.GT_ERR_STATE, A.GT_ERR_WORKSPACE,
                 A.GT_ERR_QUEUE_OVERFLOW, A.GT_ERR_TIMEOUT, A.GT_ERR_CUDA, A.GT_ERR_NO_DEVICE,
                 A.GT_ERR_UNSUPPORTED, A.GT_ERR_HOST_MEMORY):
        assert A.strerror(code) and A.strerror(code) != "unknown error"
    assert A.strerror(12345) == "unknown error"


def test_null_arguments_rejected_without_device(lib):
    from paper_2509_15377_gb300 import avalanche as A
    assert lib.gt_create(None, 0) == A.GT_ERR_ARG
    assert lib.gt_destroy(None) == A.GT_OK
    assert lib.gas_table_upload(None, None) == A.GT_ERR_ARG
    assert lib.field_setup(None, None) == A.GT_ERR_ARG
    assert lib.avalanche_run(None, None, None, None, 0, None, None) == A.GT_ERR_ARG
    assert lib.avalanche_observables(None, None, 0, 0, None, 0, 0, 0.0, None, None) == A.GT_ERR_ARG


def test_create_reports_missing_device(lib):
    import torch
    from paper_2509_15377_gb300 import avalanche as A
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.gt_create(C.byref(h), 0) == A.GT_ERR_NO_DEVICE
    with pytest.raises(A.GtError):
        A.Avalanche(0)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2509_15377_gb300 import avalanche as A
    saved = A._lib
    A._lib = None
    try:
        with pytest.raises(RuntimeError):
            A.load(str(tmp_path / "missing.so"))
    finally:
        A._lib = saved


def test_grid_maps_of_the_wrong_shape_are_refused():
    """The binding refuses a grid map that is not [nz, ny, nx, 4] (the
    kernels read one float4 per node) before touching the device."""
    from paper_2509_15377_gb300 import avalanche as A
    av = A.Avalanche.__new__(A.Avalanche)  # no device: the check comes first
    for shape in ((4, 4, 4, 3), (4, 4, 4), (1, 4, 4, 4)):
        with pytest.raises(ValueError):
            av.set_field(W.Field(W.GRID, grid=np.zeros(shape, np.float32)))


def test_primaries_of_unequal_lengths_are_refused():
    """The binding refuses primaries whose arrays differ in length (or a
    per-avalanche field of the wrong length) before anything is copied."""
    from paper_2509_15377_gb300 import avalanche as A
    av = A.Avalanche.__new__(A.Avalanche)  # no device: the check comes first
    w = W.plate(n_avalanches=6, e_field=40_000.0, seed=1)
    av.check_primaries(w.primaries)
    for key in ("dx", "aval", "uid"):
        p = W.plate(n_avalanches=6, e_field=40_000.0, seed=1).primaries
        setattr(p, key, getattr(p, key)[:-1])
        with pytest.raises(ValueError):
            av.primaries_device(p)
        with pytest.raises(ValueError):
            av.primaries_pinned(p)
    p = W.plate(n_avalanches=6, e_field=40_000.0, seed=1).primaries
    p.aval_field = np.full(p.n_avalanches - 1, 40_000.0)
    with pytest.raises(ValueError):
        av.primaries_device(p)


def test_gas_arrays_of_the_wrong_length_are_refused():
    """The binding refuses a gas whose per-level arrays do not match the
    rate table's levels, before the library reads them."""
    import dataclasses
    from paper_2509_15377_gb300 import avalanche as A
    g = W.argon_like_gas()
    for name in ("level_type", "threshold"):
        bad = dataclasses.replace(g, **{name: np.asarray(getattr(g, name))[:-1]})
        with pytest.raises(ValueError):
            A.gas_table_upload(None, bad)
    with pytest.raises(ValueError):
        A.gas_table_upload(None, dataclasses.replace(g, rate=np.asarray(g.rate).ravel()))
