"""The bounded device-side waits give up, report DG_ERR_TIMEOUT and leave the
GPU usable (dg_selftest_wait makes each kind of wait run out on purpose: an
mbarrier nothing arrives on, the same while holding tensor memory, a counter
one CTA of a cooperative launch never advances)."""
import ctypes

import numpy as np
import pytest

from paper_1805_01443_gb300 import dg, inputs


def test_selftest_rejects_unknown_kinds():
    """Refused on the host before any CUDA call (runs without a GPU)."""
    L = dg.lib()
    assert L.dg_selftest_wait(3, None) == dg.DG_ERR_ARG
    assert L.dg_selftest_wait(-1, None) == dg.DG_ERR_ARG


def _fresh_handle_steps():
    with dg.Disc(inputs.disc_planet(32, 2)) as d:
        d.step(2)
        d.sync()
        assert d.get_time()[2] == 2
        assert np.isfinite(d.fetch()).all()


@pytest.mark.gpu
def test_mbarrier_wait_times_out_and_the_gpu_stays_usable():
    L = dg.lib()
    freed = ctypes.c_int(-1)
    assert L.dg_selftest_wait(0, ctypes.byref(freed)) == dg.DG_ERR_TIMEOUT
    assert freed.value == 0
    _fresh_handle_steps()


@pytest.mark.gpu
def test_wait_holding_tensor_memory_times_out_and_frees_it():
    L = dg.lib()
    freed = ctypes.c_int(-1)
    assert L.dg_selftest_wait(1, ctypes.byref(freed)) == dg.DG_ERR_TIMEOUT
    assert freed.value == 1
    # the tensor-core inference (which allocates tensor memory) runs afterwards
    cfg = inputs.shock_ring(24, 2)
    with dg.Disc(cfg) as d:
        net = dg.Mlp(5 * 4 * 9, seed=3)
        try:
            d.set_indicator(net, 0.0)
            z, f = d.indicator_logits()
            assert np.isfinite(z).all() and f.shape == z.shape
        finally:
            net.close()


@pytest.mark.gpu
def test_counter_wait_between_ctas_times_out():
    L = dg.lib()
    assert L.dg_selftest_wait(2, None) == dg.DG_ERR_TIMEOUT
    _fresh_handle_steps()
