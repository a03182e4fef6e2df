"""The learned-initial-guess pipeline end to end on a small grid: base flows
from the plain start, network training, Newton from the prediction."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns2d  # noqa: E402
from paper_1804_03859_gb300 import learned_guess  # noqa: E402

pytestmark = pytest.mark.gpu


def test_pipeline_on_a_small_grid():
    args = learned_guess.parse(["--nx", "32", "--ny", "16", "--train", "8", "--test", "2", "--width", "4",
                                "--iters", "60", "--batch", "4", "--sfd-steps", "100", "--max-newton", "20",
                                "--chains", "3"])
    res = learned_guess.run(args)
    json.dumps(res)
    assert res["train_samples"] >= 6
    assert np.isfinite(res["unet"]["loss_last"]) and res["unet"]["loss_last"] < res["unet"]["loss_first"]
    assert res["converged"]["learned"] == res["test_samples"] == 2
    for row in res["rows"]:
        assert row["learned"]["residual"] <= 1e-10


def test_trained_network_saves_newton_work():
    """What the learned start gains over the method without it: on held-out
    (Re, D) at 64x32 the network's prediction, as Newton's start, needs fewer
    Jacobian products in total than the plain start (SFD from rest), and
    converges at least as often."""
    args = learned_guess.parse(["--nx", "64", "--ny", "32", "--train", "48", "--test", "4", "--width", "8",
                                "--iters", "800", "--batch", "16", "--sfd-steps", "150", "--max-newton", "25",
                                "--chains", "8", "--seed", "3"])
    res = learned_guess.run(args)
    rows = res["rows"]
    assert res["converged"]["learned"] >= res["converged"]["plain"]
    cap = args.max_newton * args.gmres_m * 3   # a failed solve counts as its whole budget
    cost = {k: sum(r[k]["matvecs"] if r[k]["ok"] else cap for r in rows) for k in ("plain", "learned")}
    assert cost["learned"] < cost["plain"], cost


def test_features_mark_the_cylinder():
    f = learned_guess.features(128, 64, Re=60.0, D=1.0)
    assert f.shape == (3, 64, 128)
    iy, ix = np.unravel_index(np.argmax(f[0]), f[0].shape)
    assert (ix, iy) == (32, 32)                    # x = 4, y = 4 on the 16 x 8 box
    assert np.allclose(f[1], (60.0 - 95.0) / 55.0) and np.all(f[2] == 0.0)
    chi = ns2d.cylinder_mask(ns2d.Config(nx=128, ny=64))
    assert f[0][chi > 0.5].min() > np.exp(-1.0) - 1e-12   # the bump covers the body
