"""The learned warm start: trained on solver output, it must beat the random start it replaces."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_training_and_gain(S):
    from paper_2402_08134_gb300 import warmstart as WS

    out = WS.experiment(n=3000, d=16, c=8, k=8, l=26, q=2, sweeps=60, n_train=16, n_test=3, epochs=20,
                        lr=2e-3, train_seeds=500, test_seeds=0)
    losses = out["losses"]
    assert losses[-1] < 0.8 * losses[0]
    gain = lambda key: np.median([r["random"][key] / r["learned"][key] for r in out["rows"]])  # noqa: E731
    # the learned start fits X better than the scaled random start at the first sweep and
    # keeps the lead over the early sweeps; after the sweeps both starts sit in (possibly
    # different) local minima, and the learned one must not be a worse one by more than 10%
    assert gain("obj0") > 1.0, out["rows"]
    assert gain("obj5") > 1.0, out["rows"]
    for r in out["rows"]:
        assert r["learned"]["nr"] <= 1.1 * r["random"]["nr"], (r["learned"]["nr"], r["random"]["nr"])
