"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each pin is a plain function of an ``oracle.Oracle`` so that the planted-
mistake test at the bottom can run the same pins on deliberately broken
builds of ``oracle.c`` and check that at least one of them fails.

What pins what:
* fft                -- numpy.fft (library routine), the O(N^2) DFT matrix
                        written from the definition, round trip, Parseval,
                        linearity; lengths that are not powers of two
                        (3, 5, 6, 7, 12, 96, 100, 1000) against numpy.fft.
* compress_lines, rda at lengths that are not powers of two -- the circulant
                        matrix products at those lengths.
* matched_filter     -- direct O(N*Nc) DFT sum of the centred chirp.
* compress_lines     -- circular cross-correlation with the centred chirp,
                        written as a circulant matrix product (no FFT).
* corner_turn        -- numpy transpose.
* rda                -- separable brute-force 2-D circular correlation
                        (Sec. IV-A steps 1-4 as one formula); exact
                        point-target peak value n_ca*n_cr at the planted
                        position; impulse response in closed form.
* rcmc               -- band-limited exponentials shifted by the analytic
                        fractional migration; zero Doppler unchanged.
* rda_full           -- a migrating point target focuses at its planted
                        position with the closed-form phase-only gain
                        N_cr sqrt(K_a) T, and not without RCMC.
* quality metrics    -- Dirichlet kernel (sampled sinc) closed form
                        PSLR -13.26 dB / ISLR -9.68 dB; unweighted LFM at
                        TBP >= 128 within 0.15 dB of it; low-TBP LFM against
                        the brute-force chirp autocorrelation.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

RNG = np.random.default_rng(12345)


def crand(*shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dft_matrix(n, sign=-1):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


def centred_line(chirp, n):
    """The chirp placed on a length-n line, sample j at (j - n_c/2) mod n."""
    line = np.zeros(n, np.complex128)
    m = np.arange(chirp.size) - chirp.size // 2
    np.add.at(line, m % n, chirp)
    return line


def circulant_corr_matrix(chirp, n):
    """C[p, q] = conj(line[(p - q) mod n]):  (x @ C)[q] = sum_p x[p] conj(line[p - q])."""
    line = centred_line(chirp, n)
    p = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    return np.conj(line[(p - q) % n])


# ---------------------------------------------------------------------------
# pins (each raises AssertionError on a mismatch)
# ---------------------------------------------------------------------------

def pin_fft_numpy(o):
    for n in [1, 2, 4, 8, 16, 32, 64, 128, 256, 1024, 4096]:
        x = crand(n)
        for inv in (False, True):
            ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
            got = o.fft(x, inverse=inv)
            err = np.max(np.abs(got - ref)) / max(1.0, np.max(np.abs(ref)))
            assert err < 1e-13, (n, inv, err)


def pin_fft_any_length(o):
    """Lengths that are not powers of two take the definition's O(n^2) sum."""
    for n in [3, 5, 6, 7, 12, 96, 100, 1000]:
        x = crand(n)
        for inv in (False, True):
            ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
            got = o.fft(x, inverse=inv)
            err = np.max(np.abs(got - ref)) / max(1.0, np.max(np.abs(ref)))
            assert err < 1e-12, (n, inv, err)


def pin_compress_any_length(o):
    """Line and scene compression at lengths that are not powers of two: the
    circular correlation at that length, as circulant matrix products."""
    for n, (nc, tbp) in [(100, (24, 8.0)), (96, (32, 16.0)), (300, (40, 20.0))]:
        c = sarsim.lfm_chirp(nc, tbp)
        H = o.matched_filter(n, c)
        x = crand(3, n)
        ref = x @ circulant_corr_matrix(c, n)
        got = o.compress_lines(x, H)
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)), n
    n_az, n_r = 90, 150
    ca, cr = sarsim.lfm_chirp(20, 6.0), sarsim.lfm_chirp(30, 10.0)
    raw = crand(n_az, n_r)
    img = o.rda(raw, o.matched_filter(n_r, cr), o.matched_filter(n_az, ca))
    ref = (circulant_corr_matrix(ca, n_az).T @ raw @ circulant_corr_matrix(cr, n_r)).T
    assert M.rel_l2(img, ref) < 1e-13


def pin_fft_dft_matrix(o):
    for n in [2, 4, 8, 16, 32, 64]:
        x = crand(n)
        for sign, inv in ((-1, False), (1, True)):
            ref = dft_matrix(n, sign) @ x
            err = np.max(np.abs(o.fft(x, inverse=inv) - ref)) / np.max(np.abs(ref))
            assert err < 1e-12, (n, inv, err)


def pin_fft_identities(o):
    n = 2048
    x, y = crand(n), crand(n)
    X = o.fft(x)
    # round trip
    back = o.fft(X, inverse=True) / n
    assert np.max(np.abs(back - x)) < 1e-13 * np.max(np.abs(x)) * 10
    # Parseval: sum |x|^2 = (1/N) sum |X|^2
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / n) < 1e-11 * np.sum(np.abs(x) ** 2)
    # linearity
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = o.fft(a * x + b * y)
    rhs = a * X + b * o.fft(y)
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(rhs))
    # impulse -> constant, constant -> N * impulse
    d = np.zeros(n, complex)
    d[0] = 1
    assert np.allclose(o.fft(d), np.ones(n), atol=1e-15)
    assert np.allclose(o.fft(np.ones(n)), n * d, atol=1e-9)


def pin_matched_filter(o):
    for n, (nc, tbp) in [(256, (64, 32.0)), (512, (64, 16.0)), (1024, (512, 256.0))]:
        c = sarsim.lfm_chirp(nc, tbp)
        m = np.arange(nc) - nc // 2
        k = np.arange(n)
        ref = np.conj(np.exp(-2j * np.pi * np.outer(k, m) / n) @ c)
        got = o.matched_filter(n, c)
        assert np.max(np.abs(got - ref)) < 1e-10 * nc, (n, nc)


def pin_compress_lines_circulant(o):
    n = 256
    c = sarsim.lfm_chirp(64, 32.0)
    H = o.matched_filter(n, c)
    x = crand(5, n)
    got = o.compress_lines(x, H)
    ref = x @ circulant_corr_matrix(c, n)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    # any spectrum H: y = IFFT(FFT(x) H) = circular convolution with h = IFFT(H)
    Hr = crand(n)
    h = np.fft.ifft(Hr)
    got2 = o.compress_lines(x, Hr)
    p = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    conv = h[(q - p) % n]          # y[q] = sum_p x[p] h[q - p]
    assert np.max(np.abs(got2 - x @ conv)) < 1e-11 * np.max(np.abs(got2))


def pin_corner_turn(o):
    for rows, cols in [(1, 1), (3, 5), (64, 32), (17, 130)]:
        a = crand(rows, cols)
        assert np.array_equal(o.corner_turn(a), a.T)


def pin_rda_bruteforce(o):
    spec = sarsim.scene_256()
    raw = sarsim.echo(spec)
    ca = sarsim.lfm_chirp(*spec.az_chirp)
    cr = sarsim.lfm_chirp(*spec.range_chirp)
    Hr = o.matched_filter(spec.n_range, cr)
    Ha = o.matched_filter(spec.n_az, ca)
    img = o.rda(raw, Hr, Ha)
    A = circulant_corr_matrix(ca, spec.n_az)      # [m, a]
    R = circulant_corr_matrix(cr, spec.n_range)   # [n, r]
    ref = (A.T @ raw.astype(np.complex128) @ R).T   # image[r][a]
    assert M.rel_l2(img, ref) < 1e-13
    # non-square, zero-padded azimuth (n_az < l_az)
    n_az, n_r, l_az = 100, 128, 128
    raw2 = crand(n_az, n_r)
    ca2, cr2 = sarsim.lfm_chirp(32, 8.0), sarsim.lfm_chirp(16, 8.0)
    Ha2 = o.matched_filter(l_az, ca2)
    Hr2 = o.matched_filter(n_r, cr2)
    img2 = o.rda(raw2, Hr2, Ha2, l_az=l_az)
    pad = np.zeros((l_az, n_r), complex)
    pad[:n_az] = raw2
    ref2 = (circulant_corr_matrix(ca2, l_az).T @ pad @ circulant_corr_matrix(cr2, n_r)).T[:, :n_az]
    assert img2.shape == (n_r, n_az)
    assert M.rel_l2(img2, ref2) < 1e-13


def pin_point_target_peaks(o):
    # noise-free fp64 echo: the peak is exactly n_ca * n_cr at the planted spot
    spec = sarsim.SceneSpec(512, 1024, [(100, 200), (400, 700), (300, 1000)],
                            (128, 64.0), (64, 16.0), None, 7)
    raw = sarsim.echo(spec, dtype=np.complex128)
    Hr = o.matched_filter(1024, sarsim.lfm_chirp(128, 64.0))
    Ha = o.matched_filter(512, sarsim.lfm_chirp(64, 16.0))
    img = o.rda(raw, Hr, Ha, nthreads=3)
    for (a0, r0) in spec.targets:
        assert M.peak(img, (r0, a0)) == (r0, a0)
        assert abs(img[r0, a0] - 128 * 64) < 1e-9 * 128 * 64


def pin_impulse_response(o):
    n_az, n_r = 64, 128
    a0, r0 = 10, 100
    ca, cr = sarsim.lfm_chirp(16, 4.0), sarsim.lfm_chirp(32, 16.0)
    raw = np.zeros((n_az, n_r), complex)
    raw[a0, r0] = 1.0
    img = o.rda(raw, o.matched_filter(n_r, cr), o.matched_filter(n_az, ca))
    la, lr = centred_line(ca, n_az), centred_line(cr, n_r)
    r = np.arange(n_r)[:, None]
    a = np.arange(n_az)[None, :]
    ref = np.conj(la[(a0 - a) % n_az]) * np.conj(lr[(r0 - r) % n_r])
    assert np.max(np.abs(img - ref)) < 1e-13


GEO_PIN = sarsim.Geometry(kappa=10.0, v_s=0.6, r_near=2000.0)   # ~6 range cells of migration


def pin_rcmc_bandlimited_shift(o):
    """RCMC moves each range-Doppler column by the fractional migration;
    on band-limited exponentials exp(2 pi i nu k) the Hann-windowed sinc must
    reproduce the analytic value at the fractional source position (within
    the passband ripple of a 16-tap Hann-windowed sinc, which grows with the
    frequency), and the zero-Doppler column (no migration) must come out
    unchanged up to the rounding of sin(pi t) at integers."""
    geo = GEO_PIN
    n_range = 256
    n = np.arange(n_range)[:, None]
    for n_f in (64, 63):   # an odd width: bins j >= (n_f - 1) / 2 + 1 are negative frequencies
        j = np.arange(n_f)
        f = np.where(j < n_f // 2, j, j - n_f) / n_f
        D = np.sqrt(1 - (f / (geo.kappa * geo.v_s)) ** 2)
        for nu, tol in ((0.05, 1e-3), (-0.2, 2e-3), (0.3, 5e-3)):
            rd = np.exp(2j * np.pi * nu * n) * np.ones((1, n_f))
            out = o.rcmc(rd, geo, taps=16)
            src = n + (geo.r_near + n) * (1.0 / D[None, :] - 1.0)
            exact = np.exp(2j * np.pi * nu * src)
            inside = (src >= 10) & (src < n_range - 10)
            assert np.max(np.abs(out - exact)[inside]) < tol, (n_f, nu)
            assert np.max(np.abs(out[:, 0] - rd[:, 0])) < 1e-14
        assert np.max(src - n) > 5.0      # the migration spans several range cells


def pin_rda_full_point_target(o):
    """A point target with range migration focuses at its planted position
    with the closed-form gain of the phase-only azimuth filter,
    N_cr * sqrt(K_a) * T (K_a = kappa v_s^2 / r0, T the aperture in lines),
    and RCMC is what makes it focus (without it the peak drops)."""
    geo = GEO_PIN
    n_az, n_r, ap = 1024, 256, 512
    a0, n0 = 500, 100
    raw = sarsim.echo_migration(n_az, n_r, [(a0, n0)], (64, 32.0), ap, geo, None, 1, np.complex128)
    Hr = o.matched_filter(n_r, sarsim.lfm_chirp(64, 32.0))
    img = o.rda_full(raw, Hr, geo, taps=16, nthreads=4)
    ka = geo.kappa * geo.v_s ** 2 / (geo.r_near + n0)
    ideal = 64 * np.sqrt(ka) * ap
    assert M.peak(img, (n0, a0)) == (n0, a0)
    assert abs(abs(img[n0, a0]) / ideal - 1.0) < 0.06, abs(img[n0, a0]) / ideal
    plain = o.rda_full(raw, Hr, geo, taps=0, nthreads=4)
    assert abs(plain).max() < 0.8 * abs(img[n0, a0])


ALL_PINS = [pin_fft_numpy, pin_fft_any_length, pin_compress_any_length, pin_fft_dft_matrix, pin_fft_identities,
            pin_matched_filter,
            pin_compress_lines_circulant, pin_corner_turn, pin_rda_bruteforce,
            pin_point_target_peaks, pin_impulse_response, pin_rcmc_bandlimited_shift, pin_rda_full_point_target]


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.default())


# ---------------------------------------------------------------------------
# quality metrics
# ---------------------------------------------------------------------------

def test_metrics_sinc_closed_form():
    # ideal band-limited point response: a Dirichlet kernel (rect spectrum)
    for n, frac in [(256, 0.5), (4096, 0.125), (1024, 0.25)]:
        X = np.zeros(n, complex)
        m = int(frac * n)
        X[: m // 2] = 1
        X[-(m // 2):] = 1
        s = np.fft.ifft(X) * n
        pslr, islr = M.lobe_ratios(s, 0)
        assert abs(pslr - (-13.2619)) < 0.02, pslr
        assert abs(islr - (-9.68)) < 0.02, islr


def test_lfm_high_tbp_matches_sinc():
    o = oracle.default()
    n = 4096
    for nc, tbp in [(512, 256.0), (1024, 128.0)]:
        c = sarsim.lfm_chirp(nc, tbp)
        x = np.zeros(n, complex)
        x[(np.arange(nc) - nc // 2 + 1000) % n] = c
        y = o.compress_lines(x[None], o.matched_filter(n, c))[0]
        pslr, islr = M.lobe_ratios(y, 1000)
        assert abs(pslr + 13.26) < 0.15, pslr
        assert abs(islr + 9.68) < 0.15, islr


def test_lfm_low_tbp_matches_autocorrelation():
    """At TBP 16-32 the LFM spectrum's Fresnel ripple moves PSLR away from
    the sinc value, so the expected value is the brute-force autocorrelation
    of the sampled chirp: y[d] = sum_m c(m) conj(c(m - d))."""
    o = oracle.default()
    n = 256
    for nc, tbp in [(64, 32.0), (64, 16.0)]:
        c = sarsim.lfm_chirp(nc, tbp)
        line = centred_line(c, n)
        ref = np.array([np.sum(line * np.conj(np.roll(line, d))) for d in range(n)])
        y = o.compress_lines(line[None], o.matched_filter(n, c))[0]
        assert np.max(np.abs(y - ref)) < 1e-10 * nc
        p1, i1 = M.lobe_ratios(y, 0)
        p2, i2 = M.lobe_ratios(ref, 0)
        assert abs(p1 - p2) < 1e-6 and abs(i1 - i2) < 1e-6
        assert -15.0 < p1 < -13.0


def test_snr_noise_power_estimate():
    # |n|^2 of circular complex Gaussian noise is exponential: median = ln2 * mean
    z = sarsim.complex_gaussian(3, sarsim.STREAM_NOISE, 1 << 20, 0.1).astype(np.complex128)
    assert abs(M.noise_power(z) / 0.1 - 1.0) < 0.01


def test_rel_l2_and_peak_tiebreak():
    a = np.zeros((8, 8), complex)
    a[2, 3] = 1
    a[5, 1] = 1                # equal magnitude: lowest linear index wins
    assert M.peak(a, (4, 4), window=4) == (2, 3)
    assert M.rel_l2(a, a) == 0.0
    assert abs(M.rel_l2(a * (1 + 1e-3), a) - 1e-3) < 1e-12


# ---------------------------------------------------------------------------
# planted mistakes: every deliberately broken oracle must fail a pin
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_planted_mistake_is_caught(plant, tmp_path):
    path = oracle.build(str(tmp_path / f"liboracle_plant{plant}.so"), plant=plant, force=True)
    o = oracle.Oracle(oracle.load(path))
    assert o.planted() == plant
    failed = []
    for pin in ALL_PINS:
        try:
            pin(o)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"planted mistake {plant} passed every pin"
