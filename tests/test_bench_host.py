"""Host-side checks of the benchmark's workload table and input recipes (CPU
only): every workload names a generator of ``synth`` and a preconditioner
the library knows, the blurred variants resolve their taps, and the
blurred-detector data generator keeps shapes, seeds and the row structure."""
import numpy as np

import bench
import synth

KINDS = {"none", "fourier", "mod_fourier", "haar", "block", "block_fourier", "block_haar"}


def test_workload_table():
    assert bench.WORKLOAD in bench.WORKLOADS
    for name, (builder, kind, desc, *kw) in bench.WORKLOADS.items():
        assert callable(getattr(synth, builder)), name
        assert kind in KINDS, name
        assert desc, name
        if kw:
            opts = dict(kw[0])
            noise = opts.pop("noise", None)
            assert noise is None or 0.0 < noise < 0.99
            blur = opts.pop("blur", None)
            if blur is not None:
                taps = synth.BLUR_TAPS[blur]
                assert len(taps) % 2 == 1 and len(taps) <= 7
                assert abs(sum(taps) - 1.0) < 1e-12


def test_blurred_data_recipe():
    prob = synth.config1()
    taps = synth.BLUR_TAPS["r3"]
    a = synth.with_detector_blur(prob, taps)
    b = synth.with_detector_blur(prob, taps)
    assert a.y.shape == prob.y.shape
    assert np.array_equal(a.y, b.y)                      # seeded
    assert np.all(a.y >= 0) and np.all(a.y == np.round(a.y))
    # each detector row keeps its total up to Poisson noise, less the weight
    # that cell j sends past the row ends (taps b_k with j - k outside)
    n_u = prob.geom.n_u
    r = len(taps) // 2
    kept = np.array([sum(b for k, b in zip(range(-r, r + 1), taps) if 0 <= j - k < n_u) for j in range(n_u)])
    rows = prob.y.reshape(-1, n_u)
    want = rows @ kept
    got = a.y.reshape(-1, n_u).sum(axis=1)
    assert np.all(np.abs(got - want) < 6 * np.sqrt(want) + 1)
    # a single tap of one is no blur (up to the Poisson redraw)
    c = synth.with_detector_blur(prob, [1.0])
    assert np.allclose(c.y.mean(), prob.y.mean(), rtol=1e-3)
