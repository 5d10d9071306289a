"""eaadc_ladder_noalloc: the DF ladder for callers that cannot allocate device
memory at the point of the call (their device memory already belongs to their
own memory manager, or a cudaFree's device-wide synchronisation would stall
their other streams).  It works in one fixed device array of the library
instead of allocating.

Checked through the C ABI against eaadc_ladder on the same inputs, on two
calls in a row (the second with a different vector count, so it meets the
array as the first call left it).  The ladder tests compare with the FP64
oracle to 2e-2 of max |ladder|; these two entry points share their BF16
operands and differ only in how the sum over auxiliary functions is cut into
blocks (FP32 summation order), so they are held to 1e-4 of max |ladder|.
The file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

from synth import config_problem, make_problem

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def E():
    import __graft_entry__ as g

    g.build()
    import paper_2511_05897_gb300 as mod

    return mod


class _Pool:
    """Used-memory counters of the device's default stream-ordered memory pool
    (the one eaadc_ladder allocates from), read through the driver API."""
    USED_CURRENT, USED_HIGH = 7, 8

    def __init__(self, device=0):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), device) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        val = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(val)) == 0
        return val.value

    def reset_high(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, C.byref(zero)) == 0


def _ladder_pair(E, ctx, o, v, dim, nvec, seed, pool):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    x = torch.tensor(np.random.default_rng(seed).standard_normal((nvec, dim)), device="cuda:0")
    ref = torch.empty((nvec, o, v, v), dtype=torch.float32, device="cuda:0")
    got = torch.full((nvec, o, v, v), float("nan"), dtype=torch.float32, device="cuda:0")
    E.eaadc_ladder(ctx, 0, nvec, x.data_ptr(), ref.data_ptr(), stream)
    torch.cuda.synchronize()
    used = pool.get(pool.USED_CURRENT)
    pool.reset_high()
    E.eaadc_ladder_noalloc(ctx, 0, nvec, x.data_ptr(), got.data_ptr(), stream)
    torch.cuda.synchronize()
    # nothing was taken from the stream-ordered pool during the call
    assert pool.get(pool.USED_HIGH) == used == pool.get(pool.USED_CURRENT)
    ref, got = ref.cpu().numpy(), got.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


@pytest.mark.parametrize("o,v,naux,decay,seed,calls", [
    (20, 200, 600, 150.0, 1, (2, 1)),   # o=20, v=200, naux=600: the sum over Q runs in several blocks
    (2, 70, 30, 10.0, 3, (3, 1)),       # v=70 is not a multiple of 8: padded intermediate and staged result
])
def test_ladder_noalloc_matches_ladder(E, o, v, naux, decay, seed, calls):
    pr = config_problem("canonical-200") if (o, v, naux) == (20, 200, 600) else make_problem(o, v, naux, decay, seed)
    ctx = E.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_canonical(ctx, 3, 1.0)
        dim = E.eaadc_state_info(ctx, 0)[2]
        pool = _Pool(0)
        for i, nvec in enumerate(calls):
            _ladder_pair(E, ctx, o, v, dim, nvec, seed + 10 * i, pool)
    finally:
        E.eaadc_destroy(ctx)


def test_ladder_noalloc_rejects_what_does_not_fit(E):
    """Too many vectors for the fixed array, or no BF16 operands yet: a clear
    error status, nothing launched."""
    import torch

    pr = config_problem("canonical-200")
    ctx = E.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_canonical(ctx, 3, 1.0)
        dim = E.eaadc_state_info(ctx, 0)[2]
        o, v = pr["o"], pr["v"]
        x = torch.zeros((9, dim), dtype=torch.float64, device="cuda:0")
        out = torch.zeros((9, o, v, v), dtype=torch.float32, device="cuda:0")
        stream = torch.cuda.current_stream().cuda_stream
        with pytest.raises(E.EaadcError) as err:
            E.eaadc_ladder_noalloc(ctx, 0, 1, x.data_ptr(), out.data_ptr(), stream)
        assert err.value.status == E.EAADC_ERR_STATE and "BF16 operands" in str(err.value)
        E.eaadc_ladder(ctx, 0, 1, x.data_ptr(), out.data_ptr(), stream)  # makes the BF16 operands
        with pytest.raises(E.EaadcError) as err:
            E.eaadc_ladder_noalloc(ctx, 0, 9, x.data_ptr(), out.data_ptr(), stream)
        assert err.value.status == E.EAADC_ERR_ARG and "fixed limit" in str(err.value)
        E.eaadc_ladder_noalloc(ctx, 0, 8, x.data_ptr(), out.data_ptr(), stream)  # 8 vectors fit
        torch.cuda.synchronize()
        assert not out[:8].any()
    finally:
        E.eaadc_destroy(ctx)
