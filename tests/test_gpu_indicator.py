"""The learned troubled-cell indicator end to end on the shock-ring disc (P3,
128^2): labels from the TVB test on the method's own run, training with
libdg's kernels, then on held-out runs (other seeds) the miss and false-flag
rates against the TVB test, and the solution the network-limited run gives
against the TVB-limited one, next to what no troubled-cell limiting gives:
the network must keep most of what the TVB limiter does."""
import pytest

from paper_1805_01443_gb300 import indicator, inputs

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")


def test_learned_indicator_on_the_shock_ring():
    rec = indicator.evaluate(inputs.shock_ring(128, 3, seed=5), inputs.shock_ring(128, 3, seed=6),
                             inputs.shock_ring(128, 3, seed=7), snapshots=12, every=4, epochs=80,
                             err_steps=30)
    print(rec)
    assert rec["troubled"] > 100
    assert rec["miss_rate"] <= 0.05
    assert rec["false_flag_rate"] <= 0.05
    e_mlp = rec["runs"]["mlp"]["rel_l2_sigma_vs_tvb"]
    e_none = rec["runs"]["none"]["rel_l2_sigma_vs_tvb"]
    assert e_none > 0
    assert e_mlp < 0.25 * e_none
