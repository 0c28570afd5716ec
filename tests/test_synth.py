"""Host-side checks of the seeded workload generator (no GPU)."""
import numpy as np

from paper_2507_14046_gb300 import synth


def test_splitmix64_known_answer():
    # first output of SplitMix64 from state 0 (Steele et al. 2014 reference implementation)
    z = synth._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_counter_based_streams_are_offset_consistent():
    a = synth.normal(7, 3, 100)
    b = synth.normal(7, 3, 40, offset=30)
    np.testing.assert_array_equal(a[60:100], b)
    u = synth.uniform(1, 2, 200000)
    assert 0.0 < u.min() and u.max() < 1.0
    z = synth.normal(1, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_workload_shapes_and_phantom():
    w = synth.SINGLE_16
    J = synth.sensitivity_raw(w.grid, w.rings, 0)
    assert J.shape == (208, 2048) and J.dtype == np.float32
    truth = synth.sequence_truth(w)
    assert truth.shape == (1, 2048)
    vals = np.unique(truth)
    np.testing.assert_array_equal(vals, [-0.3, 0.0])
    amp = synth.breathing_amplitude(20)
    assert amp[15] == 0.0 and np.isclose(amp[5], 1.0)
    V = synth.measurements(J, truth, 0)
    assert V.shape == (1, 208)
    Zin = synth.input_noise(2048, 8, 0)
    assert Zin.shape == (2048, 8) and abs(Zin.std() - 0.1) < 0.005


def test_measurement_snr():
    J = synth.sensitivity_raw((16, 16, 8), 1, 0)
    truth = synth.sequence_truth(synth.SINGLE_16)
    clean = synth.measurements(J, truth, 0, snr_db=400.0)
    noisy = synth.measurements(J, truth, 0, snr_db=40.0)
    snr = 20 * np.log10(np.sqrt(np.mean(clean.astype(np.float64) ** 2))
                        / np.sqrt(np.mean((noisy - clean).astype(np.float64) ** 2)))
    assert abs(snr - 40.0) < 1.5


def test_random_ellipsoids_inside_grid_and_batch_shapes():
    shapes = synth.batch_problem_shapes(64, 1)
    assert len(shapes) == 64
    assert {g for g, _ in shapes} <= set(synth.BATCH_GRIDS)
    for p, (g, r) in enumerate(shapes[:8]):
        for e in synth.random_ellipsoids(g, 1, p):
            for a in range(3):
                assert 2.0 <= e.semi[a] <= 8.0
                assert e.centre[a] - e.semi[a] >= -1e-12
                assert e.centre[a] + e.semi[a] <= g[a] + 1e-12
