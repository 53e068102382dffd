"""Algorithmic traffic and FLOP conventions used to report the kernels.

* FFT FLOP convention (Table I of the paper): an N-point complex FFT counts
  5 N log2 N flops; GFLOPS = 5 N log2 N / t.
* Fused line compression (Sec. II-B): two transforms plus the spectrum
  multiply, 2 * 5 N log2 N + 6 N flops per line.
* Algorithmic HBM bytes: a fused pass reads and writes every complex64
  sample once (16 bytes per sample, Sec. II-B: two transfers per line); the
  corner turn also reads and writes every sample once.  Filters and twiddles
  (at most 128 KiB, reused by every line from L2) are not counted.

Pure host arithmetic; importing this module needs neither torch nor a GPU.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import re

C64 = 8  # bytes per complex64 sample
_HERE = os.path.dirname(os.path.abspath(__file__))


def fft_flops(n: int) -> float:
    return 5.0 * n * math.log2(n)


def fft_gflops(n: int, seconds_per_fft: float) -> float:
    return fft_flops(n) / seconds_per_fft / 1e9


def fused_line_flops(n: int) -> float:
    return 2.0 * fft_flops(n) + 6.0 * n


def fused_pass_bytes(n_lines: int, n: int) -> int:
    return 2 * C64 * n_lines * n


def corner_turn_bytes(rows: int, cols: int) -> int:
    return 2 * C64 * rows * cols


def rda_bytes(n_az: int, n_range: int) -> int:
    """Three passes (range, corner turn, azimuth): 48 bytes per sample."""
    return fused_pass_bytes(n_az, n_range) + corner_turn_bytes(n_az, n_range) + fused_pass_bytes(n_range, n_az)


def rda_bytes_folded(n_az: int, n_range: int) -> int:
    """Corner turn folded into the range pass: 32 bytes per sample."""
    return fused_pass_bytes(n_az, n_range) + fused_pass_bytes(n_range, n_az)


def rda_flops(n_az: int, n_range: int) -> float:
    return n_az * fused_line_flops(n_range) + n_range * fused_line_flops(n_az)


def _local_includes(path: str, seen: set) -> None:
    """`path` and every csrc file it includes with #include "...", recursively."""
    if path in seen or not os.path.exists(path):
        return
    seen.add(path)
    with open(path) as fh:
        for line in fh:
            m = re.match(r'\s*#\s*include\s+"([^"]+)"', line)
            if m:
                _local_includes(os.path.normpath(os.path.join(os.path.dirname(path), m.group(1))), seen)


def _code_only(text: str) -> str:
    """C/C++ source without its comments, whitespace runs collapsed to one
    blank: what the compiler sees, so that a comment edit leaves it alone."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":                         # string or character literal, kept whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def kernel_source_hash(root: str | None = None) -> str:
    """sha256 over the code (comments and whitespace left out) of the CUDA
    sources of the kernels whose traffic is recorded: the 4096-point schedule
    table (the fused and folded range-pass kernels) and every header it
    includes; a recorded ncu traffic figure is valid only for this hash.
    `root`: the package directory to read (this one by default)."""
    h = hashlib.sha256()
    seen: set = set()
    _local_includes(os.path.join(root or _HERE, "csrc", "sched_4096.cu"), seen)
    for f in sorted(seen):
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, profiles_dir: str) -> int | None:
    """DRAM bytes per launch recorded by ncu for `key` ("fused <schedule>" or
    "range_ct <schedule>"), or None if absent or recorded for other kernel
    sources."""
    try:
        with open(os.path.join(profiles_dir, "ncu_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    ent = rec.get("kernels", {}).get(key)
    return int(ent["bytes"]) if ent else None
