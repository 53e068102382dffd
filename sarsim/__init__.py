"""Seeded synthetic SAR scenes: the one input module that both the oracle
and the CUDA path consume.

It holds no compression arithmetic (no FFT, no filter, no correlation).  It
only draws random numbers, evaluates the point-target signal model and writes
complex64 echo matrices, following the simulator described in Sec. V-A of
the paper (point targets, chirp signal model, additive Gaussian noise) with
the normalised parameters below, because the paper does not give its sampling
rate, PRF or pulse lengths.

Signal model
------------
* Reference chirp (linear FM, unit amplitude, no window) of ``n_c`` samples
  and time-bandwidth product ``tbp``:  c(m) = exp(i pi K m^2) for
  m = -n_c/2 ... n_c/2 - 1 with K = tbp / n_c^2 cycles/sample^2, i.e. a
  bandwidth of tbp / n_c of the sampling rate.
* A target at (a0, r0) adds c_a(ma) * c_r(mr) at azimuth row (a0 + ma) mod N_a
  and range column (r0 + mr) mod N_r: the chirp is centred on the target, so
  the compressed peak lands exactly on (a0, r0) with value n_ca * n_cr.
* Noise: circular complex Gaussian of total variance 10^(-snr_db/10) relative
  to the unit chirp amplitude (real and imaginary parts each half of it).

Random numbers
--------------
Counter-based: the i-th 64-bit value of stream ``s`` under seed ``S`` is
splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser as published by Vigna) applied to the
counter  key(S, s) + (i + 1) * 0x9E3779B97F4A7C15, where
key(S, s) = splitmix64(S xor (s * 0xD1B54A32D192ED03)).  Uniforms on [0, 1)
take the top 53 bits; normals use the Box-Muller transform.  Any consumer can
regenerate value i alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
STREAM_MUL = 0xD1B54A32D192ED03
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

STREAM_TARGETS = 1
STREAM_NOISE = 2


def splitmix64(z):
    """splitmix64 finaliser on uint64 (array or scalar), wrapping arithmetic."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    s = np.uint64((int(seed) ^ (int(stream) * STREAM_MUL)) & 0xFFFFFFFFFFFFFFFF)
    return np.uint64(splitmix64(s))


def random_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    key = stream_key(seed, stream)
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = key + (i + np.uint64(1)) * GOLDEN
    return splitmix64(ctr)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles on [0, 1) from the top 53 bits."""
    return (random_u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def complex_gaussian(seed: int, stream: int, count: int, variance: float,
                     chunk: int = 1 << 22) -> np.ndarray:
    """``count`` circular complex normals of total variance ``variance``.

    Sample j uses uniforms 2j and 2j+1 of the stream (Box-Muller: the first
    drives the radius, the second the angle)."""
    out = np.empty(count, np.complex64)
    sd = np.sqrt(variance / 2.0)
    for s in range(0, count, chunk):
        n = min(chunk, count - s)
        u = uniform(seed, stream, 2 * s, 2 * n)
        u1 = 1.0 - u[0::2]          # (0, 1]
        u2 = u[1::2]
        rad = np.sqrt(-2.0 * np.log(u1)) * sd
        ang = 2.0 * np.pi * u2
        out[s:s + n] = (rad * np.cos(ang) + 1j * (rad * np.sin(ang))).astype(np.complex64)
    return out


def lfm_chirp(n_c: int, tbp: float) -> np.ndarray:
    """Unit-amplitude linear FM chirp, complex128, sample j <-> time m = j - n_c/2.

    The phase pi*K*m^2 (K = tbp/n_c^2) is reduced modulo 2*pi exactly: with
    integer tbp the product tbp*m^2 is an exact integer in float64, reduced
    modulo 2*n_c^2 before scaling."""
    m = np.arange(n_c, dtype=np.float64) - (n_c // 2)
    cycles2 = np.fmod(float(tbp) * m * m, 2.0 * n_c * n_c) / float(n_c * n_c)  # phase / pi
    return np.cos(np.pi * cycles2) + 1j * np.sin(np.pi * cycles2)


@dataclass
class SceneSpec:
    n_az: int
    n_range: int
    targets: list = field(default_factory=list)      # [(a0, r0), ...]
    range_chirp: tuple = (64, 32.0)                  # (n_c, tbp)
    az_chirp: tuple = (64, 16.0)
    snr_db: float | None = 20.0                      # None: no noise
    seed: int = 1
    l_az: int | None = None                          # azimuth transform length (>= n_az)

    @property
    def az_len(self) -> int:
        return self.l_az if self.l_az else self.n_az


def place_targets(seed: int, n_az: int, n_range: int, count: int, margin_az: int = 64,
                  margin_r: int = 64, min_sep: int = 256, max_tries: int = 100000) -> list:
    """Seeded target positions: azimuth uniform in [margin_az, n_az - margin_az),
    range uniform in [margin_r, n_range - margin_r), pairwise Chebyshev distance
    >= min_sep (rejection sampling; draw i uses uniforms 2i and 2i+1 of the
    target stream).  The separation is relaxed for scenes too small to hold
    ``count`` targets that far apart."""
    sep = min(min_sep, max(1, min(n_az, n_range) // (2 * max(count, 1))))
    if 2 * margin_az >= n_az or 2 * margin_r >= n_range:
        raise ValueError("place_targets: margins leave no room")
    out, i = [], 0
    while len(out) < count and i < max_tries:
        u = uniform(seed, STREAM_TARGETS, 2 * i, 2)
        i += 1
        a = margin_az + int(u[0] * (n_az - 2 * margin_az))
        r = margin_r + int(u[1] * (n_range - 2 * margin_r))
        if all(max(abs(a - pa), abs(r - pr)) >= sep for pa, pr in out):
            out.append((a, r))
    if len(out) < count:
        raise ValueError("place_targets: could not place the targets")
    return out


def echo(spec: SceneSpec, dtype=np.complex64) -> np.ndarray:
    """The n_az x n_range raw echo of ``spec`` (targets + noise), complex64 by
    default; ``dtype=np.complex128`` keeps the noise-free signal unrounded."""
    n_az, n_r = spec.n_az, spec.n_range
    sig = np.zeros((n_az, n_r), np.complex128)
    ca = lfm_chirp(*spec.az_chirp)
    cr = lfm_chirp(*spec.range_chirp)
    rows_off = np.arange(len(ca)) - len(ca) // 2
    cols_off = np.arange(len(cr)) - len(cr) // 2
    patch = np.outer(ca, cr)
    for (a0, r0) in spec.targets:
        rows = (a0 + rows_off) % n_az
        cols = (r0 + cols_off) % n_r
        sig[np.ix_(rows, cols)] += patch
    if spec.snr_db is not None:
        var = 10.0 ** (-spec.snr_db / 10.0)
        noise = complex_gaussian(spec.seed, STREAM_NOISE, n_az * n_r, var)
        sig += noise.reshape(n_az, n_r).astype(np.complex128)
    return sig.astype(dtype)


# ---------------------------------------------------------------------------
# The named workloads.
# ---------------------------------------------------------------------------

def scene_256() -> SceneSpec:
    """256 x 256, one target at (128, 128), range LFM 64 / TBP 32, azimuth
    LFM 64 / TBP 16, 20 dB SNR, seed 1."""
    return SceneSpec(256, 256, [(128, 128)], (64, 32.0), (64, 16.0), 20.0, 1)


def scene_4096(seed: int = 2) -> SceneSpec:
    """4096 x 4096, five seeded targets, range LFM 512 / TBP 256, azimuth
    LFM 1024 / TBP 128, 10 dB SNR, seed 2."""
    tg = place_targets(seed, 4096, 4096, 5)
    return SceneSpec(4096, 4096, tg, (512, 256.0), (1024, 128.0), 10.0, seed)


def scaled_chirps(n_range: int, l_az: int) -> tuple:
    """Chirps scaled to a strip's size, keeping the 4096^2 scene's ratios:
    range n_c = N_r/8 with TBP n_c/2, azimuth n_c = L/4 with TBP n_c/8."""
    ncr = max(8, n_range // 8)
    nca = max(8, l_az // 4)
    return (ncr, ncr / 2.0), (nca, nca / 8.0)


def next_pow2(n: int) -> int:
    return 1 << (int(n) - 1).bit_length()


def strip_spec(seed: int, n_range: int, n_az: int, n_targets: int, snr_db: float = 10.0) -> SceneSpec:
    """A strip of a ragged batch: azimuth transform length L = max(256, next
    power of two >= n_az), chirps scaled to the strip (the azimuth chirp no
    longer than the strip), seeded targets kept at least half a chirp from
    every edge where the strip is tall enough, so that no echo wraps."""
    l_az = max(256, next_pow2(n_az))
    (ncr, tbr), (nca, tba) = scaled_chirps(n_range, l_az)
    if nca > n_az:
        nca = n_az
        tba = nca / 8.0
    m_az = nca // 2 + 1
    m_r = ncr // 2 + 1
    if 2 * m_az >= n_az:
        m_az = 0
    tg = place_targets(seed, n_az, n_range, n_targets, margin_az=m_az, margin_r=m_r,
                       min_sep=min(256, max(1, n_az // 4)))
    return SceneSpec(n_az, n_range, tg, (ncr, tbr), (nca, tba), snr_db, seed, l_az=l_az)


STREAM_BATCH = 3
STREAM_REQUESTS = 5


def ragged_batch_specs(seed: int = 4, count: int = 64) -> list:
    """The ragged batch: `count` strips, range length drawn from {1024, 2048,
    4096, 8192, 16384}, azimuth line count uniform in [256, 4096], 1 to 8
    targets, chirps scaled to each strip; strip i uses uniforms 3i .. 3i+2 of
    the batch stream and its own seed for targets and noise."""
    u = uniform(seed, STREAM_BATCH, 0, 3 * count)
    out = []
    for i in range(count):
        n_range = 1024 << int(u[3 * i] * 5)
        n_az = 256 + int(u[3 * i + 1] * (4096 - 256 + 1))
        n_t = 1 + int(u[3 * i + 2] * 8)
        out.append(strip_spec(seed * 1000 + i, n_range, n_az, n_t))
    return out


SERVING_SIZES = (2048, 4096, 8192, 16384)
SERVING_MIX = (0.70, 0.25, 0.04, 0.01)


def serving_requests(seed: int = 5, n: int = 2000, variants: int = 2) -> list:
    """Size class and scene variant of each of n requests: size drawn with
    probabilities SERVING_MIX over SERVING_SIZES (uniform 2i of the request
    stream), variant uniform over `variants` (uniform 2i+1).  Returns
    [(size_index, variant), ...]."""
    u = uniform(seed, STREAM_REQUESTS, 0, 2 * n)
    edges = np.cumsum(SERVING_MIX)
    out = []
    for i in range(n):
        k = int(np.searchsorted(edges, u[2 * i], side="right"))
        out.append((min(k, len(SERVING_SIZES) - 1), int(u[2 * i + 1] * variants)))
    return out


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """n arrival times (seconds) of a Poisson process of `rate` per second:
    exponential gaps -ln(1 - u)/rate from stream 6."""
    u = uniform(seed, 6, 0, n)
    return np.cumsum(-np.log1p(-u) / rate)


def serving_scene(size: int, variant: int, seed: int = 5) -> SceneSpec:
    """Pool scene of a serving size class: 1 to 16 seeded targets, chirps
    scaled as for the strips (range n/8 with TBP n/16, azimuth n/4 with TBP
    n/32), 10 dB SNR."""
    s = seed * 100 + variant * 10 + SERVING_SIZES.index(size) if size in SERVING_SIZES else seed * 100 + variant
    n_t = 1 + int(uniform(s, STREAM_TARGETS, 10 ** 6, 1)[0] * 16)
    rc, ac = scaled_chirps(size, size)
    tg = place_targets(s, size, size, n_t, margin_az=ac[0] // 2 + 1, margin_r=rc[0] // 2 + 1,
                       min_sep=min(256, size // 32))
    return SceneSpec(size, size, tg, rc, ac, 10.0, s)


# ---------------------------------------------------------------------------
# Range-migration scenes (full Range-Doppler processing with RCMC).
# ---------------------------------------------------------------------------

@dataclass
class Geometry:
    """Normalised side-looking geometry, in range samples and azimuth lines.

    kappa:  two-way phase in cycles per range sample of path (2 dr / lambda);
    v_s:    platform displacement per azimuth line, in range samples;
    r_near: slant range of range bin 0, in range samples.
    A target at range bin n0 and azimuth line a0 has closest range
    r0 = r_near + n0 and range history r(m) = sqrt(r0^2 + v_s^2 (m - a0)^2);
    its azimuth chirp rate is kappa v_s^2 / r0 cycles per line^2."""
    kappa: float = 10.0
    v_s: float = 0.3
    r_near: float = 4000.0

    def as_tuple(self):
        return (self.kappa, self.v_s, self.r_near)


def echo_migration(n_az: int, n_range: int, targets: list, range_chirp: tuple, aperture: int, geo: Geometry,
                   snr_db: float | None, seed: int, dtype=np.complex64) -> np.ndarray:
    """Raw echo with range migration: target (a0, n0) contributes, on each
    azimuth line m with |m - a0| < aperture/2, the range chirp delayed to the
    fractional range r(m) - r_near,
        exp(i pi K (n - (r(m) - r_near))^2)  for |n - (r(m) - r_near)| < n_c/2,
    times the two-way phase exp(-2 pi i kappa r(m)).  Lines and range samples
    do not wrap.  Noise as in `echo`."""
    n_c, tbp = range_chirp
    K = tbp / (n_c * n_c)
    sig = np.zeros((n_az, n_range), np.complex128)
    n = np.arange(n_range, dtype=np.float64)
    for (a0, n0) in targets:
        r0 = geo.r_near + n0
        for m in range(max(0, a0 - aperture // 2), min(n_az, a0 + aperture - aperture // 2)):
            r = np.sqrt(r0 * r0 + (geo.v_s * (m - a0)) ** 2)
            t = n - (r - geo.r_near)
            on = (t >= -(n_c // 2)) & (t < n_c - n_c // 2)
            cyc = np.fmod(geo.kappa * r, 1.0)
            sig[m, on] += np.exp(1j * np.pi * K * t[on] * t[on]) * np.exp(-2j * np.pi * cyc)
    if snr_db is not None:
        var = 10.0 ** (-snr_db / 10.0)
        sig += complex_gaussian(seed, STREAM_NOISE, n_az * n_range, var).reshape(n_az, n_range).astype(np.complex128)
    return sig.astype(dtype)


def migration_scene_4096(seed: int = 2):
    """The 4096 x 4096 scene of the full processor: the five targets of
    scene_4096 (range bins and lines), range LFM 512 / TBP 256, synthetic
    aperture 1024 lines, geometry kappa 10, v_s 0.3, r_near 4000 (about 3.5
    range cells of migration at the aperture edges), 10 dB SNR.  Returns
    (targets, range_chirp, aperture, geometry, snr_db, seed)."""
    base = scene_4096(seed)
    return base.targets, (512, 256.0), 1024, Geometry(10.0, 0.3, 4000.0), 10.0, seed
