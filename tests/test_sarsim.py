"""The seeded input generator: published known answers, determinism, the
statistics it promises and the signal model's geometry."""
import numpy as np

import sarsim


def test_splitmix64_known_answers():
    # splitmix64 from state 0: the first outputs of the published generator
    g = sarsim.GOLDEN
    with np.errstate(over="ignore"):
        assert int(sarsim.splitmix64(g)) == 0xE220A8397B1DCDAF
        assert int(sarsim.splitmix64(g * np.uint64(2))) == 0x6E789E6AA1B965F4
        assert int(sarsim.splitmix64(g * np.uint64(3))) == 0x06C45D188009454F


def test_counter_based_random_access():
    a = sarsim.random_u64(9, 2, 0, 1000)
    b = sarsim.random_u64(9, 2, 500, 10)
    assert np.array_equal(a[500:510], b)
    assert not np.array_equal(a, sarsim.random_u64(10, 2, 0, 1000))
    assert not np.array_equal(a, sarsim.random_u64(9, 1, 0, 1000))


def test_uniform_and_gaussian_statistics():
    u = sarsim.uniform(1, 2, 0, 1 << 20)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 2e-3
    z = sarsim.complex_gaussian(1, 2, 1 << 20, 0.1).astype(np.complex128)
    assert abs(np.mean(np.abs(z) ** 2) - 0.1) < 1e-3
    assert abs(np.mean(z.real ** 2) - 0.05) < 1e-3
    assert abs(np.mean(z.real * z.imag)) < 1e-3


def test_chirp_model():
    c = sarsim.lfm_chirp(64, 32.0)
    assert c.shape == (64,)
    assert np.allclose(np.abs(c), 1.0, atol=1e-15)
    m = np.arange(64) - 32
    assert np.allclose(c, np.exp(1j * np.pi * (32.0 / 64 ** 2) * m * m), atol=1e-13)
    assert c[32] == 1.0                       # m = 0


def test_echo_deterministic_and_targets():
    s = sarsim.scene_256()
    a, b = sarsim.echo(s), sarsim.echo(s)
    assert a.dtype == np.complex64 and a.shape == (256, 256)
    assert np.array_equal(a, b)
    s.snr_db = None
    clean = sarsim.echo(s, dtype=np.complex128)
    # support of the single target: 64 azimuth rows x 64 range columns
    rows = np.nonzero(np.abs(clean).sum(1))[0]
    cols = np.nonzero(np.abs(clean).sum(0))[0]
    assert rows.min() == 128 - 32 and rows.max() == 128 + 31
    assert cols.min() == 128 - 32 and cols.max() == 128 + 31


def test_scene_4096_targets():
    t = sarsim.scene_4096().targets
    assert len(t) == 5
    for i, (a, r) in enumerate(t):
        assert 64 <= a < 4096 - 64 and 64 <= r < 4096 - 64
        for (a2, r2) in t[i + 1:]:
            assert max(abs(a - a2), abs(r - r2)) >= 256
    assert t == sarsim.scene_4096().targets


def test_strip_spec():
    s = sarsim.strip_spec(4, 2048, 700, 5)
    assert s.l_az == 1024 and s.n_az == 700
    assert s.range_chirp == (256, 128.0) and s.az_chirp == (256, 32.0)
    for (a, r) in s.targets:
        assert 129 <= a < 700 - 129
