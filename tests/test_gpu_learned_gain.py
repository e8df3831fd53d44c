"""What the trained boundary network gains over the open edge without it.

A short training run (solver-generated trajectories on 3x enlarged periodic domains, the
library's own forward/backward/Adam kernels) must cut the reflected fraction of a pulse leaving
an open grid well below that of the zero-incoming edge, against a light-cone-enlarged FP64
periodic reference."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_reflects_less_than_zero_incoming(gpu_lib):
    from paper_1601_08103_gb300 import learned_boundary as lb

    lee = gpu_lib
    x, t = lb.generate_samples(lee, trajectories=192, region=64, steps=128, record_every=2, batch=96, seed=21)
    assert x.shape[0] > 10000
    params, hist = lb.train(lee, x, t, steps=1500, batch_rows=4096, lr=3e-3, lr_final=2e-4, seed=1, log_every=500)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    ev = lb.evaluate(lee, params, n=256, steps=600, sample_every=20, seed=5)
    zero = ev["forms"]["zero"]["reflected_fraction"]
    learned = ev["forms"]["learned"]["reflected_fraction"]
    assert np.isfinite(learned)
    assert learned < 0.5 * zero, ev
