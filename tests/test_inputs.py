"""The seeded input recipes: reproducible, seed-dependent, and shaped as the
workloads state (no arithmetic of the method lives in them)."""
import numpy as np

from paper_1805_01443_gb300 import inputs


def test_modal_perturbation_is_seeded_and_decays_with_degree():
    shape = (3, 16, 8, 8)
    a = inputs.modal_perturbation(shape, seed=4, amp=1e-3)
    assert np.array_equal(a, inputs.modal_perturbation(shape, seed=4, amp=1e-3))
    assert not np.array_equal(a, inputs.modal_perturbation(shape, seed=5, amp=1e-3))
    m = 4
    for k in range(16):
        bound = 1e-3 * 0.5 ** (k // m + k % m)
        assert np.abs(a[:, k]).max() <= bound
        assert np.abs(a[:, k]).max() > 0.5 * bound  # uniform on (-bound, bound)


def test_batched_workload_recipe():
    """48 discs: sizes 128/256/384/512 and degrees 2/3/4 cycling, planet mass
    10^U(-6, -4) from each instance's own seed, damping zones on."""
    a = inputs.batch_discs()
    b = inputs.batch_discs()
    assert len(a) == 48
    qs = [c["planet"]["q"] for c in a]
    assert qs == [c["planet"]["q"] for c in b]
    assert all(1e-6 <= q <= 1e-4 for q in qs) and len(set(qs)) == 48
    for k, c in enumerate(a):
        assert c["mesh"]["nx"] == c["mesh"]["ny"] == (128, 256, 384, 512)[k % 4]
        assert c["order"] == (2, 3, 4)[k % 3]
        assert c["disc"]["seed"] == 100 + k and c["disc"]["rdamp_in"] > 0 and c["disc"]["rdamp_out"] > 0
    # an instance's draw depends on its seed only, not on its place in the batch
    assert inputs.batch_discs(n=5, seed0=103)[0]["planet"]["q"] == qs[3]


def test_benchmark_disc_recipe():
    """P4 512x512 on [-2.5, 2.5]^2, locally isothermal h = 0.05, Sigma ~ r^-1/2,
    planet q = 3e-5 at r_p = 1 with eps = 0.6 h, damping radii 0.4 / 2.1."""
    c = inputs.disc_planet_512()
    assert c["order"] == 4 and c["mesh"]["nx"] == c["mesh"]["ny"] == 512
    assert (c["mesh"]["x0"], c["mesh"]["x1"]) == (-2.5, 2.5)
    assert c["eos"]["kind"] == 0 and c["eos"]["h"] == 0.05
    assert c["disc"]["sigma_slope"] == -0.5 and c["disc"]["rk"] == 3
    assert c["planet"]["q"] == 3e-5 and c["planet"]["enabled"] == 1
    assert abs(c["planet"]["eps"] - 0.03) < 1e-15
    assert (c["disc"]["rdamp_in"], c["disc"]["rdamp_out"]) == (0.4, 2.1)
