"""Batched precision form (dg_batch_*): many discs of mixed size and degree in
one launch per stage, against each disc stepped on its own with dg_step.

The batched kernels run the same per-tile code on the same data in the same
per-instance order of reductions, so the results are compared bit for bit.
"""
import numpy as np
import pytest

from paper_1805_01443_gb300 import dg, inputs

pytestmark = pytest.mark.gpu


def make(cfgs):
    return [dg.Disc(c) for c in cfgs]


def close(ds):
    for d in ds:
        d.close()


def assert_same(a, b):
    np.testing.assert_array_equal(a.fetch(), b.fetch())
    assert a.get_time() == b.get_time()
    np.testing.assert_array_equal(a.torque_series(), b.torque_series())


def test_batch_equals_individual_steps():
    cfgs = inputs.batch_small()
    solo, bat = make(cfgs), make(cfgs)
    try:
        for d in solo:
            d.step(7)
        with dg.Batch(bat) as b:
            b.step(3)
            b.step(4)
            b.sync()
        for a, c in zip(bat, solo):
            assert_same(a, c)
    finally:
        close(solo + bat)


@pytest.mark.parametrize("policy,dynamic,ctas", [(0, 1, 0), (1, 1, 0), (2, 1, 0), (1, 0, 0), (2, 1, 1)])
def test_batch_schedules_give_identical_results(policy, dynamic, ctas):
    cfgs = inputs.batch_small()
    ref, bat = make(cfgs), make(cfgs)
    try:
        for d in ref:
            d.step(5)
        with dg.Batch(bat) as b:
            b.config(policy, dynamic, ctas)
            b.step(5)
        for a, c in zip(bat, ref):
            assert_same(a, c)
    finally:
        close(ref + bat)


def test_batch_tune_does_not_advance_and_then_matches():
    cfgs = inputs.batch_small()
    ref, bat = make(cfgs), make(cfgs)
    try:
        for d in ref:
            d.step(2)
        for d in bat:
            d.step(2)
        u0 = [d.fetch() for d in bat]
        with dg.Batch(bat) as b:
            best = b.tune(steps=2)
            assert best["policy"] in (0, 1, 2) and best["ms_per_step"] > 0
            for d, u in zip(bat, u0):
                np.testing.assert_array_equal(d.fetch(), u)
                assert d.get_time()[2] == 2
            b.step(4)
        for d in ref:
            d.step(4)
        for a, c in zip(bat, ref):
            assert_same(a, c)
    finally:
        close(ref + bat)


def test_handles_continue_after_batched_steps():
    """Odd batched step counts flip each handle's ping-pong buffers; dg_step,
    dg_set_state and a second batch afterwards see the right state."""
    cfgs = inputs.batch_small()[:3]
    ref, bat = make(cfgs), make(cfgs)
    try:
        for d in ref:
            d.step(3)
        with dg.Batch(bat) as b:
            b.step(3)
        for d in bat + ref:
            d.step(2)
        for a, c in zip(bat, ref):
            assert_same(a, c)
        u = ref[0].fetch()
        t = ref[0].get_time()
        bat[0].set_state(u, t[0], t[2])
        ref[0].set_state(u, t[0], t[2])
        with dg.Batch(bat) as b:
            b.step(1)
        for d in ref:
            d.step(1)
        for a, c in zip(bat, ref):
            assert_same(a, c)
    finally:
        close(ref + bat)


def test_batch_rejects_fp64_and_bad_counts():
    fp64 = dg.Disc(inputs.disc_small(16, 2))
    try:
        with pytest.raises(dg.DgError) as e:
            dg.Batch([fp64])
        assert e.value.code == dg.DG_ERR_UNSUPPORTED
        with pytest.raises(dg.DgError) as e:
            dg.Batch([])
        assert e.value.code == dg.DG_ERR_ARG
    finally:
        fp64.close()
