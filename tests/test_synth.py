"""The seeded input generator: SplitMix64 published outputs, ranges, recipes."""
import numpy as np

from paper_1803_02977_gb300 import synth


def test_splitmix64_reference_outputs():
    # outputs of the published SplitMix64 reference generator (Steele, Lea &
    # Flood 2014; the widely used C version of the same constants)
    assert [int(v) for v in synth.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert int(synth.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_counter_based_offsets():
    a = synth.splitmix64(77, 100)
    b = synth.splitmix64(77, 40, start=60)
    assert np.array_equal(a[60:], b)


def test_noise_surface_range_and_perimeter():
    h = synth.noise_surface(33, 17, 5)
    assert h.shape == (17, 33)
    inner = h[1:-1, 1:-1]
    assert inner.min() >= 0.0 and inner.max() < 1.0
    assert np.all(h[0] == 0) and np.all(h[-1] == 0) and np.all(h[:, 0] == 0) and np.all(h[:, -1] == 0)
    assert np.array_equal(h, synth.noise_surface(33, 17, 5))


def test_south_tilt():
    flat = synth.noise_surface(8, 10, 2)
    tilt = synth.noise_surface(8, 10, 2, south_tilt=1e-4, dx=100.0)
    d = tilt[1:-1, 1:-1] - flat[1:-1, 1:-1]
    # 1e-4 m/m over 100 m cells: 0.01 m per row, falling toward row ny-1
    assert np.allclose(d[:, 0], 0.01 * np.arange(8, 0, -1))


def test_batch_workload_draws():
    b = synth.batch_workload()
    assert b.count == 512
    assert min(b.sides) >= 128 and max(b.sides) <= 1024
    assert all(1e-6 <= k <= 1e-4 for k in b.K)
    assert all(0.4 <= m <= 0.6 for m in b.m)
    assert b.seeds[0] == 1000 and b.seeds[-1] == 1511
