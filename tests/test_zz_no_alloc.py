"""avalanche_run_static: the batched run with the library's fixed internal
scratch instead of a caller work space, for callers that cannot allocate
device memory where they run avalanches.  Its results must equal
avalanche_run's (the same kernels, the same random numbers), on two calls in
a row through the same array, and the second call must leave the device's
free memory and torch's allocations unchanged.

This file is collected last on purpose (test_zz_*), and it also passes on
its own in a fresh process: it builds and creates everything it uses."""
import ctypes as C

import numpy as np
import pytest

from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import assert_same_electrons

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def av():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    a = A.Avalanche(0)
    yield a
    a.close()


def _fetch(av, n):
    return av.fetch(n)


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
def test_static_scratch_matches_workspace_run(av, precision):
    import torch
    w = W.plate(n_avalanches=48, e_field=45_000.0, seed=31)
    av.set_gas(w.gas)
    av.set_field(w.field)
    prim = av.primaries_device(w.primaries)
    opt = A.RunOptions(seed=31, t_max=0.35, precision=precision)
    cap = 200_000
    stream = torch.cuda.current_stream(0)
    # reference: the existing entry point with a caller-provided work space
    st_ref = av.run(prim, opt, cap, stream=stream, allow=(A.GT_OK,))
    ref = _fetch(av, st_ref["n_endpoints"])
    # the same run twice through the fixed internal scratch (the second call
    # reuses the array the first one left behind)
    r = av.make_run(prim, opt)
    out = av.endpoints_struct(cap)
    for call in range(2):
        if call == 1:
            # after the first call (which may load the device code): the
            # device's free memory and torch's allocations stay as they are
            free0, alloc0 = torch.cuda.mem_get_info(0)[0], torch.cuda.memory_allocated(0)
        st = A.avalanche_run_static(av.ctx, r, out, stream.cuda_stream, allow=(A.GT_OK,))
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info(0)[0] == free0
            assert torch.cuda.memory_allocated(0) == alloc0
        got = _fetch(av, st.n_endpoints)
        assert st.n_endpoints == st_ref["n_endpoints"]
        assert st.real_collisions == st_ref["real_collisions"]
        assert_same_electrons(got, ref, scale_pos=w.field.gap, scale_t=0.35)
        assert np.array_equal(got["electrons"], ref["electrons"])
        assert np.array_equal(got["tallies"], ref["tallies"])


def test_static_scratch_limits_are_enforced(av):
    w = W.plate(n_avalanches=4, seed=32)
    av.set_gas(w.gas)
    av.set_field(w.field)
    lib = A.load()
    st = A.gt_stats()
    # capacity beyond the fixed array
    prim = av.primaries_device(w.primaries)
    r = av.make_run(prim, A.RunOptions(seed=32, t_max=0.05))
    av.alloc(A.GT_STATIC_MAX_ELECTRONS + 1, r.n_avalanches, r)
    out = av.endpoints_struct(A.GT_STATIC_MAX_ELECTRONS + 1)
    assert lib.avalanche_run_static(av.ctx, C.byref(r), C.byref(out), None,
                                    C.byref(st)) == A.GT_ERR_WORKSPACE
    # host-memory primaries are not accepted (no staging space is reserved)
    hp = av.primaries_pinned(w.primaries)
    rh = av.make_run(hp, A.RunOptions(seed=32, t_max=0.05))
    out = av.endpoints_struct(1000)
    assert lib.avalanche_run_static(av.ctx, C.byref(rh), C.byref(out), None,
                                    C.byref(st)) == A.GT_ERR_ARG
