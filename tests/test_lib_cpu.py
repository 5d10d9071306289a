"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point declared in include/eaadc.h, and
rejects bad arguments with a status instead of aborting."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g

    g.build()
    import paper_2511_05897_gb300 as E

    return E


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "eaadc.h")).read()
    return sorted(set(re.findall(r"\b(eaadc_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(built):
    E = built
    L = E.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(E.EXPORTED)
    assert "sm_103a" in E.eaadc_version()


def test_bad_arguments_return_status(built):
    E = built
    ctx = C.c_void_p()
    z = np.zeros(4)
    st = E.lib().eaadc_init(C.byref(ctx), 0, 2, 1, E._lib._dp(z), E._lib._dp(z), E._lib._dp(z), 0, None)
    assert st == E.EAADC_ERR_ARG
    assert ctx.value is None
    assert "invalid" in E.eaadc_last_error(None)
    assert E.lib().eaadc_build_canonical(None, 3, 1.0) == E.EAADC_ERR_ARG
    E.eaadc_destroy(None)


def test_no_silent_cpu_fallback(built):
    """Without a usable GPU the library reports a CUDA error; it never computes on the host."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    E = built
    with pytest.raises(E.EaadcError) as ei:
        E.eaadc_init(1, 1, 1, np.array([-1.0]), np.array([1.0]), np.ones((1, 2, 2)), 0)
    assert ei.value.status in (E.EAADC_ERR_CUDA, E.EAADC_ERR_ARG)
