"""FP64 reference Range-Doppler compressor (the oracle) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library
(``paper_2604_03585_gb300``) never imports, links or calls it, and the two
share no code: the only module both sides use is ``sarsim``, the seeded input
generator, which holds none of the compression arithmetic.

The arithmetic lives in plain C (``oracle.c``), compiled with gcc into
``oracle/_build/liboracle.so`` and called here through ``ctypes`` on numpy
complex128 arrays.  What each function computes, and the passage of the paper
it follows, is stated in ``oracle.c``.

Pins: every function here is checked by ``tests/test_oracle_pins.py`` against
numpy's FFT and brute-force DFT matrices, Parseval, linearity, brute-force
circulant correlation, closed-form point-target peaks, impulse responses and
the closed-form PSLR/ISLR of an unweighted LFM (see ``oracle.metrics``).
The paper's own Table IV quality values cannot be pinned: its scene is not
fully specified (parity unpinned for those values only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(out_path: str | None = None, plant: int = 0, force: bool = False) -> str:
    """Compile oracle.c with gcc into a shared library and return its path.

    ``plant`` > 0 builds a variant carrying one deliberate mistake (used only
    by the test that checks the pins catch it).  No -ffast-math, and FMA
    contraction is off so that x86-64 and aarch64 builds round identically.
    """
    out_path = out_path or _LIB_PATH
    if not force and plant == 0 and os.path.exists(out_path) and \
            os.path.getmtime(out_path) >= os.path.getmtime(_SRC):
        return out_path
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           f"-DORACLE_PLANT={int(plant)}", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, c_int, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_fft.argtypes = [i64, vp, c_int]
    lib.oracle_matched_filter.argtypes = [i64, i64, vp, vp]
    lib.oracle_compress_line.argtypes = [i64, vp, vp]
    lib.oracle_compress_lines.argtypes = [i64, i64, vp, vp, c_int]
    lib.oracle_corner_turn.argtypes = [i64, i64, vp, vp]
    lib.oracle_rda.argtypes = [i64, i64, i64, vp, vp, vp, vp, c_int]
    d = ctypes.c_double
    lib.oracle_rcmc.argtypes = [i64, i64, vp, vp, d, d, d, c_int]
    lib.oracle_rda_full.argtypes = [i64, i64, vp, vp, d, d, d, c_int, vp, c_int]
    for name in ("oracle_fft", "oracle_matched_filter", "oracle_compress_line",
                 "oracle_compress_lines", "oracle_corner_turn", "oracle_rda", "oracle_planted", "oracle_rcmc",
                 "oracle_rda_full"):
        getattr(lib, name).restype = c_int
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


class Oracle:
    """numpy front end of one build of ``oracle.c`` (the default build, or a
    planted-mistake variant in the pin tests)."""

    def __init__(self, lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else load()

    def fft(self, x, inverse: bool = False) -> np.ndarray:
        """Unnormalised DFT, X[k] = sum_n x[n] exp(-+2 pi i n k / N)."""
        y = _c128(x).copy()
        _check(self.lib.oracle_fft(y.size, _ptr(y), 1 if inverse else -1), "fft")
        return y

    def matched_filter(self, n: int, chirp) -> np.ndarray:
        """H = conj(FFT_n(chirp centred on index 0)), unnormalised."""
        c = _c128(chirp)
        H = np.empty(n, np.complex128)
        _check(self.lib.oracle_matched_filter(n, c.size, _ptr(c), _ptr(H)), "matched_filter")
        return H

    def compress_lines(self, data, H, nthreads: int = 1) -> np.ndarray:
        """Each row y = IFFT(FFT(row) . H) (fused line compression)."""
        d = _c128(data).copy()
        Hc = _c128(H)
        n = d.shape[-1]
        _check(self.lib.oracle_compress_lines(d.size // n, n, _ptr(d), _ptr(Hc), nthreads),
               "compress_lines")
        return d

    def corner_turn(self, a) -> np.ndarray:
        x = _c128(a)
        rows, cols = x.shape
        out = np.empty((cols, rows), np.complex128)
        _check(self.lib.oracle_corner_turn(rows, cols, _ptr(x), _ptr(out)), "corner_turn")
        return out

    def rda(self, raw, Hr, Ha, l_az: int | None = None, nthreads: int = 1) -> np.ndarray:
        """Range compression, corner turn, azimuth compression.

        raw is n_az x n_range; returns the n_range x n_az image.  ``l_az``
        (default n_az) is the azimuth transform length for zero-padded lines.
        """
        r = _c128(raw)
        n_az, n_range = r.shape
        l_az = n_az if l_az is None else int(l_az)
        Hr_c, Ha_c = _c128(Hr), _c128(Ha)
        if Hr_c.size != n_range or Ha_c.size != l_az:
            raise ValueError("oracle: filter lengths do not match the scene")
        img = np.empty((n_range, n_az), np.complex128)
        _check(self.lib.oracle_rda(n_az, n_range, l_az, _ptr(r), _ptr(Hr_c), _ptr(Ha_c),
                                   _ptr(img), nthreads), "rda")
        return img

    def rcmc(self, rd, geo, taps: int = 16) -> np.ndarray:
        """RCMC of range-Doppler data rd[n_range][n_f] (see oracle.c)."""
        x = _c128(rd)
        n_range, n_f = x.shape
        out = np.empty_like(x)
        _check(self.lib.oracle_rcmc(n_range, n_f, _ptr(x), _ptr(out), *geo.as_tuple(), taps), "rcmc")
        return out

    def rda_full(self, raw, Hr, geo, taps: int = 16, nthreads: int = 1) -> np.ndarray:
        """Range compression, corner turn, azimuth FFT, RCMC, range-dependent
        azimuth filter, azimuth IFFT: raw[n_az][n_range] -> image[n_range][n_az]."""
        r = _c128(raw)
        n_az, n_range = r.shape
        Hr_c = _c128(Hr)
        img = np.empty((n_range, n_az), np.complex128)
        _check(self.lib.oracle_rda_full(n_az, n_range, _ptr(r), _ptr(Hr_c), *geo.as_tuple(), taps, _ptr(img),
                                        nthreads), "rda_full")
        return img

    def planted(self) -> int:
        return int(self.lib.oracle_planted())


_default: Oracle | None = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def fft(x, inverse=False):
    return default().fft(x, inverse)


def matched_filter(n, chirp):
    return default().matched_filter(n, chirp)


def compress_lines(data, H, nthreads=1):
    return default().compress_lines(data, H, nthreads)


def corner_turn(a):
    return default().corner_turn(a)


def rda(raw, Hr, Ha, l_az=None, nthreads=1):
    return default().rda(raw, Hr, Ha, l_az, nthreads)


def rda_full(raw, Hr, geo, taps=16, nthreads=1):
    return default().rda_full(raw, Hr, geo, taps, nthreads)
