"""Image-quality metrics of a compressed SAR image -- TEST INFRASTRUCTURE ONLY.

The paper reports an L2 relative error, a maximum absolute error and a
per-target SNR (Table IV) and names PSLR and ISLR as its point-target quality
measures (Sec. I, contribution 3), without defining them.  The readings used
here:

* rel_l2(a, ref) = ||a - ref||_2 / ||ref||_2 over the whole complex image, FP64.
* peak(img, pos): argmax of |img|^2 within +-32 samples (Chebyshev) of pos;
  ties go to the lowest linear index.
* PSLR / ISLR of a target: take the cuts through its peak along each image
  axis, upsample each whole cut 16x by zero-padding its DFT, and walk outward
  from the peak to the first local minimum on each side (the mainlobe).
  PSLR = max sidelobe power / peak power; ISLR = sidelobe energy / mainlobe
  energy, over the whole cut except +-64 samples around the other targets.
  Both in dB.  An unweighted LFM compresses to a sinc: PSLR -13.26 dB and,
  over a wide window, ISLR about -9.7 dB.
* SNR of a target = 10 log10(|peak|^2 / P_n), with P_n = median(|img|^2)/ln 2
  over the whole image (|noise|^2 of circular complex Gaussian noise is
  exponential, whose median is ln 2 times its mean).
"""
from __future__ import annotations

import math
import numpy as np


def rel_l2(a, ref) -> float:
    a = np.asarray(a, np.complex128)
    ref = np.asarray(ref, np.complex128)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((a - ref).ravel()) / (den if den > 0 else 1.0))


def max_abs(a, ref) -> float:
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(ref, np.complex128))))


def peak(img, pos, window: int = 32) -> tuple:
    """(row, col) of the largest |img|^2 within +-window of pos (rows/cols wrap)."""
    img = np.asarray(img)
    R, C = img.shape
    r0, c0 = pos
    best, best_lin = -1.0, None
    for dr in range(-window, window + 1):
        r = (r0 + dr) % R
        row = np.abs(img[r].astype(np.complex128)) ** 2
        for dc in range(-window, window + 1):
            c = (c0 + dc) % C
            v = row[c]
            lin = r * C + c
            if v > best or (v == best and (best_lin is None or lin < best_lin)):
                best, best_lin = v, lin
    return (best_lin // C, best_lin % C)


def _upsample(cut: np.ndarray, factor: int) -> np.ndarray:
    """Band-limited (DFT zero-padding) upsampling of a whole periodic cut."""
    n = cut.size
    X = np.fft.fft(cut)
    Z = np.zeros(n * factor, np.complex128)
    h = n // 2
    Z[:h] = X[:h]
    Z[-(n - h):] = X[h:]
    return np.fft.ifft(Z) * factor


def lobe_ratios(cut, peak_index: int, exclude=(), factor: int = 16, exclude_half: int = 64) -> tuple:
    """(PSLR_dB, ISLR_dB) of one cut with its peak at ``peak_index``.

    ``exclude`` lists other targets' positions on this cut; +-exclude_half
    samples around each are left out of the sidelobe region."""
    cut = np.asarray(cut, np.complex128)
    n = cut.size
    up = np.abs(_upsample(cut, factor)) ** 2
    m = up.size
    # locate the upsampled peak near the sample peak
    centre = peak_index * factor
    lo, hi = centre - factor, centre + factor
    idx = np.arange(lo, hi + 1) % m
    p = int(idx[np.argmax(up[idx])])
    pk = up[p]
    # walk outward to the first local minimum on each side
    left = 0
    while left < m // 2 and up[(p - left - 1) % m] < up[(p - left) % m]:
        left += 1
    right = 0
    while right < m // 2 and up[(p + right + 1) % m] < up[(p + right) % m]:
        right += 1
    main = np.zeros(m, bool)
    main[(p + np.arange(-left, right + 1)) % m] = True
    side = ~main
    for q in exclude:
        qs = int(q) * factor
        side[(qs + np.arange(-exclude_half * factor, exclude_half * factor + 1)) % m] = False
    if not side.any():
        return float("nan"), float("nan")
    pslr = 10.0 * math.log10(up[side].max() / pk)
    islr = 10.0 * math.log10(up[side].sum() / up[main].sum())
    return pslr, islr


def noise_power(img) -> float:
    p = np.abs(np.asarray(img).astype(np.complex128)) ** 2
    return float(np.median(p) / math.log(2.0))


def snr_db(img, pos, p_n: float | None = None) -> float:
    img = np.asarray(img)
    p_n = noise_power(img) if p_n is None else p_n
    return 10.0 * math.log10(abs(complex(img[pos])) ** 2 / p_n)


def quality(img, targets_img) -> dict:
    """Per-target peak position, PSLR/ISLR along both image axes and SNR.

    ``targets_img`` are the planted (row, col) positions in image coordinates
    (for an n_range x n_az image: (r0, a0))."""
    img = np.asarray(img)
    p_n = noise_power(img)
    out = []
    for i, t in enumerate(targets_img):
        pr, pc = peak(img, t)
        others_rows = [o[0] for j, o in enumerate(targets_img) if j != i and abs(o[1] - pc) <= 64]
        others_cols = [o[1] for j, o in enumerate(targets_img) if j != i and abs(o[0] - pr) <= 64]
        ps_c, is_c = lobe_ratios(img[pr, :], pc, exclude=others_cols)
        ps_r, is_r = lobe_ratios(img[:, pc], pr, exclude=others_rows)
        out.append(dict(pos=(int(pr), int(pc)), pslr_axis1=ps_c, islr_axis1=is_c,
                        pslr_axis0=ps_r, islr_axis0=is_r, snr=snr_db(img, (pr, pc), p_n)))
    return dict(targets=out, noise_power=p_n)
