"""Batched precision form (dg_batch_*): many discs of mixed size and degree in
one launch per stage, against the FP64 oracle run of each disc and against
each disc stepped on its own with dg_step.

Against the oracle the precision form's stated bounds hold per instance
(relative L2 of Sigma and momentum <= 1e-5, of the torque series <= 1e-6,
of Sigma - Sigma_bg <= 5e-6 after 12 steps: measured at most 4e-7).
Against per-instance steps the batched kernels run the same per-tile code on
the same data in the same per-instance order of reductions, so the results are
compared bit for bit.
"""
import numpy as np
import pytest

import oracle
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


# (policy, dynamic, ctas_per_sm, tiles_per_item): persistent per-stage
# launches, one CTA per tile, and the flow schedule (one launch per step)
SCHEDULES = [(0, 1, 0, 1), (1, 1, 0, 1), (2, 1, 0, 1), (1, 0, 0, 1), (2, 1, 1, 1), (1, 2, 0, 1), (0, 2, 0, 2),
             (2, 2, 0, 4), (1, 2, 1, 4), (1, 3, 0, 1), (2, 3, 1, 2)]
ORACLE_STEPS = 12


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def oracle_runs():
    """Each instance of the small mixed batch (degrees 1-4, ragged tiles),
    ORACLE_STEPS steps of the FP64 oracle: initial and final state, torque
    series, time, and the noise-free background density."""
    cfgs = inputs.batch_small()
    runs = []
    for cfg in cfgs:
        o = oracle.Oracle(cfg)
        u0 = o.fetch()
        tq = []
        for _ in range(ORACLE_STEPS):
            o.step(1)
            tq.append(o.torque()[0])
        bg = dict(cfg, disc=dict(cfg["disc"], noise_amp=0.0))
        runs.append({"u0": u0, "u": o.fetch(), "tq": np.array(tq), "t": o.get_time(),
                     "sig_bg": oracle.Oracle(bg).fetch()[0]})
        o.close()
    return cfgs, runs


@pytest.mark.parametrize("policy,dynamic,ctas,tpi", SCHEDULES)
def test_batch_matches_the_oracle(oracle_runs, policy, dynamic, ctas, tpi):
    """Every instance of a batched run against its own FP64 oracle run, under
    every schedule of the batched launches."""
    cfgs, runs = oracle_runs
    bat = make(cfgs)
    try:
        for d, r in zip(bat, runs):
            d.set_state(r["u0"])
        with dg.Batch(bat) as b:
            b.config(policy, dynamic, ctas, tpi)
            b.step(ORACLE_STEPS)
            b.sync()
        for k, (d, r) in enumerate(zip(bat, runs)):
            ug, uo = d.fetch(), r["u"]
            assert rel(ug[0], uo[0]) <= 1e-5, k
            assert max(rel(ug[1], uo[1]), rel(ug[2], uo[2])) <= 1e-5, k
            assert rel(ug[0] - r["sig_bg"], uo[0] - r["sig_bg"]) <= 5e-6, k
            assert rel(d.torque_series(), r["tq"]) <= 1e-6, k
            t, _, st = d.get_time()
            assert st == ORACLE_STEPS
            assert abs(t - r["t"][0]) <= 1e-6 * r["t"][0], k
    finally:
        close(bat)


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


@pytest.mark.parametrize("policy,dynamic,ctas,tpi", SCHEDULES)
def test_batch_schedules_give_identical_results(policy, dynamic, ctas, tpi):
    cfgs = inputs.batch_small()
    ref, bat = make(cfgs), make(cfgs)
    try:
        for d in ref:
            d.step(5)
        with dg.Batch(bat) as b:
            b.config(policy, dynamic, ctas, tpi)
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
            assert best["dynamic"] in (0, 1, 2, 3) and best["tiles_per_item"] in (1, 2, 4)
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


def test_flow_schedule_continues_after_odd_step_counts():
    """One persistent launch per step: odd step counts, a switch of schedule in
    the middle and dg_step afterwards give the per-instance results."""
    cfgs = inputs.batch_small()[2:5]
    ref, bat = make(cfgs), make(cfgs)
    try:
        for d in ref:
            d.step(6)
        with dg.Batch(bat) as b:
            b.config(1, 2, 0, 2)
            b.step(3)
            b.config(0, 1, 0, 1)
            b.step(1)
            b.config(2, 2, 0, 1)
            b.step(1)
        for d in bat:
            d.step(1)
        for a, c in zip(bat, ref):
            assert_same(a, c)
    finally:
        close(ref + bat)


def test_batch_config_rejects_bad_schedules():
    bat = make(inputs.batch_small()[:1])
    try:
        with dg.Batch(bat) as b:
            for args in [(3, 1, 0, 1), (1, 4, 0, 1), (1, 2, 0, 3), (1, 2, -1, 1)]:
                with pytest.raises(dg.DgError) as e:
                    b.config(*args)
                assert e.value.code == dg.DG_ERR_ARG
    finally:
        close(bat)
