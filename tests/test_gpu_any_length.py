"""GPU: line lengths that are not powers of two (2 ... 8192) against the FP64
oracle, whose transform at such lengths is the DFT's definition: the exact
length-n compression y = IFFT_n(FFT_n(x) . H) (Sec. II-B) and the scene
compression (Sec. IV-A) at those lengths."""
import os

import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = max(1, os.cpu_count() or 1)
LINE_TOL = 4e-6
SCENE_TOL = 2e-5


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    torch.cuda.set_device(0)
    return sar


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def noise(seed, rows, n):
    return sarsim.complex_gaussian(seed, 0, rows * n, 1.0).reshape(rows, n)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def seven_smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


# n, lines: lengths whose prime factors are 2, 3, 5, 7 (the mixed-radix
# engine at the length itself: one to four passes, radices 2 ... 32, prime
# factors 3, 5, 7 alone and combined) and other lengths (the zero-padded
# convolution at every engine length L = max(256, next pow2 >= 2n - 1) from
# 256 to 16384), the smallest and largest n of several of them, and n = 2
@pytest.mark.parametrize("n,lines", [(2, 5), (3, 7), (6, 5), (7, 5), (12, 5), (15, 4), (49, 4), (100, 9),
                                     (128, 9), (129, 9), (255, 9), (257, 6), (343, 4), (500, 6), (1000, 5),
                                     (1023, 5), (1029, 4), (1500, 4), (2000, 3), (2049, 3), (2401, 2), (3000, 3),
                                     (3125, 2), (4000, 2), (4095, 3), (4374, 2), (5000, 2), (6000, 2), (6561, 2),
                                     (7000, 2), (7776, 2), (8000, 2), (8191, 2)])
def test_line_compression_any_length(sar, orc, n, lines):
    x = noise(31 + n, lines, n)
    nc = max(1, n // 4)
    H = orc.matched_filter(n, sarsim.lfm_chirp(nc, nc / 2.0))
    ref = orc.compress_lines(x, H, nthreads=NTHREADS)
    dummy = dev(np.ones(lines))
    plan = sar.sar_plan_create(n, lines, dev(H), dummy)
    got_d = dev(x)
    sar.sar_range_compress(plan, got_d)
    torch.cuda.synchronize()
    got = got_d.cpu().numpy()
    # any spectrum, out of place as well (not a matched filter: no symmetry to hide behind)
    Hr = noise(7, 1, n)[0]
    ref2 = orc.compress_lines(x, Hr, nthreads=NTHREADS)
    plan2 = sar.sar_plan_create(n, lines, dev(Hr), dummy)
    xd = dev(x)
    out = torch.empty_like(xd)
    sar.sar_range_compress_oop(plan2, xd, out)
    torch.cuda.synchronize()
    got2 = out.cpu().numpy()
    assert np.array_equal(xd.cpu().numpy(), x.astype(np.complex64))
    sched = sar.sar_plan_get_schedules(plan)[0]
    L = sched["n"]
    plan.destroy()
    plan2.destroy()
    e1, e2 = M.rel_l2(got, ref), M.rel_l2(got2, ref2)
    print(f"\nANY n={n} ({sched['name']}, L={L}): matched {e1:.2e}, random H {e2:.2e}")
    if seven_smooth(n):
        assert L == n and "mixed" in sched["name"]
    else:
        assert L == max(256, 1 << (2 * n - 2).bit_length())
    assert e1 < LINE_TOL and e2 < LINE_TOL


# lengths with a compile-time specialisation of the mixed-radix kernel; lines
# span several blocks and end in a partial one
@pytest.mark.parametrize("n,lines", [(1000, 13), (2000, 7), (3000, 5), (4000, 5), (5000, 3), (6000, 3),
                                     (8000, 3), (1200, 9), (1500, 5), (2400, 3), (3500, 2), (4800, 2), (7200, 2)])
def test_specialised_mixed_kernel_equals_runtime_kernel(sar, n, lines, monkeypatch):
    """The kernels compiled for one length and the runtime-radix kernels run
    the same passes on the same tables: bit-identical results, for the fused
    compression and for the plain transform both ways."""
    x = dev(noise(41 + n, lines, n))
    Hr = dev(noise(8, 1, n)[0])
    plan = sar.sar_plan_create(n, lines, Hr, dev(np.ones(lines)))
    outs = []
    for generic in ("0", "1"):
        monkeypatch.setenv("SAR_MIXED_GENERIC", generic)
        c, f, i = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        sar.sar_range_compress_oop(plan, x, c)
        sar.sar_fft_lines(n, lines, x, f, False)
        sar.sar_fft_lines(n, lines, x, i, True)
        torch.cuda.synchronize()
        outs.append((c, f, i))
    plan.destroy()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("n_az,n_range", [(300, 1000), (256, 3000), (1000, 256), (300, 4096), (33, 77)])
def test_scene_any_length_vs_oracle(sar, orc, n_az, n_range):
    """Scene compression with lengths that are not powers of two in either
    dimension (300 x 4096 folds the corner turn into the range pass with
    image rows of 300 samples)."""
    (ncr, tbr), _ = sarsim.scaled_chirps(n_range, 256)
    nca = max(4, n_az // 4)
    tba = max(1.0, nca / 8.0)
    targets = [(n_az // 4, n_range // 3), (3 * n_az // 4, 2 * n_range // 3)]
    if n_az < 100:   # one target: two would share each other's peak-search window
        targets = [(n_az // 2, n_range // 2)]
    spec = sarsim.SceneSpec(n_az=n_az, n_range=n_range, targets=targets, range_chirp=(ncr, tbr),
                            az_chirp=(nca, tba), snr_db=20.0, seed=8)
    raw = sarsim.echo(spec)
    Hr = orc.matched_filter(n_range, sarsim.lfm_chirp(ncr, tbr))
    Ha = orc.matched_filter(n_az, sarsim.lfm_chirp(nca, tba))
    ref = orc.rda(raw, Hr, Ha, nthreads=NTHREADS)
    plan = sar.sar_plan_create(n_range, n_az, dev(Hr), dev(Ha))
    img = torch.empty((n_range, n_az), dtype=torch.complex64, device="cuda")
    raw_d = dev(raw)
    sar.sar_rda_process(plan, raw_d, img)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    folded = sar.sar_plan_folds_corner_turn(plan)
    plan.destroy()
    err = M.rel_l2(got, ref)
    print(f"\nANY scene {n_az}x{n_range}: rel_l2 {err:.2e} folded={folded}")
    assert err < SCENE_TOL
    for (a0, r0) in targets:
        assert M.peak(got, (r0, a0)) == M.peak(ref, (r0, a0)) == (r0, a0)
    if n_range in (1000, 3000, 4096) and n_az % 4 == 0:
        assert folded


@pytest.mark.parametrize("n_az,n_range", [(64, 1000), (40, 1200), (64, 1500), (44, 1600), (32, 2000), (28, 2400),
                                          (48, 2500), (64, 3000), (128, 5000), (64, 8000), (32, 7200), (36, 4500)])
def test_folded_corner_turn_at_seven_smooth_lengths(sar, n_az, n_range):
    """Range lengths with a compiled mixed-radix kernel fold the corner turn
    into the range pass (groups of four lines: one block of four for
    64-thread lines, clusters of two or four blocks for 128- and 256-thread
    lines): the image equals the unfolded path's (range pass, separate corner
    turn) bit for bit."""
    x = noise(71 + n_range, n_az, n_range)
    Hr, Ha = dev(noise(72, 1, n_range)[0]), dev(noise(73, 1, n_az)[0])
    folded = sar.sar_plan_create(n_range, n_az, Hr, Ha)
    plain = sar.sar_plan_create(n_range, n_az, Hr, Ha, flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
    assert sar.sar_plan_folds_corner_turn(folded) and not sar.sar_plan_folds_corner_turn(plain)
    a = torch.empty((n_range, n_az), dtype=torch.complex64, device="cuda")
    b = torch.empty_like(a)
    sar.sar_rda_process(folded, dev(x), a)
    sar.sar_rda_process(plain, dev(x), b)
    torch.cuda.synchronize()
    folded.destroy()
    plain.destroy()
    assert torch.equal(a, b)


def test_schedules_of_any_length_plans(sar):
    a, b = dev(np.ones(1009)), dev(np.ones(300))
    plan = sar.sar_plan_create(1009, 300, a, b)       # 1009 is prime: zero-padded convolution
    r, z = sar.sar_plan_get_schedules(plan)
    assert r["n"] == 2048 and r["name"].startswith("wrap_")
    assert z["n"] == 300 and z["name"] == "n300_mixed_r20x15"   # 300 = 20 * 15: mixed radix, two passes
    assert not sar.sar_plan_folds_corner_turn(plan)
    plan.destroy()
    plan = sar.sar_plan_create(300, 1009, b, a)
    r, z = sar.sar_plan_get_schedules(plan)
    assert r["name"] == "n300_mixed_r20x15" and z["name"].startswith("wrap_")
    plan.destroy()
    # wrap and mixed-radix schedules are not part of the enumeration (never autotuned)
    assert not [d for d in sar.schedules() if d["name"].startswith("wrap_") or "mixed" in d["name"]]


def test_any_length_refusals(sar):
    a, b = dev(np.ones(1000)), dev(np.ones(256))
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(8193, 256, dev(np.ones(8193)), b)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create_ex(1000, 256, a, b, range_schedule="n1024_e32_r32x32_l4")
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    # the unfused pipeline needs a transform at the line length itself: the
    # zero-padded convolution of 1009 has none
    a9 = dev(np.ones(1009))
    plan = sar.sar_plan_create(1009, 256, a9, b)
    x = torch.zeros((256, 1009), dtype=torch.complex64, device="cuda")
    img = torch.empty((1009, 256), dtype=torch.complex64, device="cuda")
    for call in (lambda: sar.sar_range_compress_unfused(plan, x),
                 lambda: sar.sar_rda_process_unfused(plan, x, img)):
        with pytest.raises(sar.SarError) as e:
            call()
        assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    sar.sar_rda_process(plan, x, img)      # the fused path runs
    torch.cuda.synchronize()
    assert float(img.abs().max()) == 0.0
    plan.destroy()
    x = torch.zeros((256, 1000), dtype=torch.complex64, device="cuda")
    img = torch.empty((1000, 256), dtype=torch.complex64, device="cuda")
    plan = sar.sar_plan_create(256, 1000, b, a)
    sar.sar_plan_set_geometry(plan, 10.0, 0.3, 100.0, 16)
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_full(plan, x, torch.empty_like(img), torch.empty_like(img))
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    plan.destroy()


@pytest.mark.parametrize("n_az,n_range", [(256, 1000), (300, 3000)])
def test_unfused_pipeline_at_seven_smooth_lengths(sar, orc, n_az, n_range):
    """The unfused comparison pipeline (DFT kernel, spectrum multiply, inverse
    DFT kernel) at a 7-smooth range length runs on the mixed-radix engine's
    plain transform: the same image as the fused path, to rounding."""
    x = noise(61 + n_range, n_az, n_range)
    Hr = orc.matched_filter(n_range, sarsim.lfm_chirp(n_range // 8, n_range / 16.0))
    Ha = orc.matched_filter(n_az, sarsim.lfm_chirp(64, 16.0))
    plan = sar.sar_plan_create(n_range, n_az, dev(Hr), dev(Ha))
    a = dev(x)
    b = dev(x)
    sar.sar_range_compress(plan, a)
    sar.sar_range_compress_unfused(plan, b)
    torch.cuda.synchronize()
    ref = orc.compress_lines(x, Hr, nthreads=NTHREADS)
    assert M.rel_l2(a.cpu().numpy(), ref) < LINE_TOL
    assert M.rel_l2(b.cpu().numpy(), ref) < LINE_TOL
    plan.destroy()


# ---------------------------------------------------------------------------
# the DFT itself at any length (the mixed-radix engine at 7-smooth lengths,
# Bluestein on the power-of-two engine at the others)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 100, 127, 128, 255, 1000, 3000, 5000, 8191])
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_fft_any_length_vs_oracle(sar, orc, n, inverse):
    """sar_fft_lines at lengths that are not powers of two (or below 256)
    against the oracle's DFT, which at such lengths is the definition's sum."""
    x = noise(97 + n, 3, n)
    ref = np.stack([orc.fft(row, inverse=inverse) for row in x])
    xd = dev(x)
    out = torch.empty_like(xd)
    sar.sar_fft_lines(n, 3, xd, out, inverse)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    err = M.rel_l2(got, ref)
    print(f"\nDFT n={n} {'inv' if inverse else 'fwd'}: rel_l2 {err:.2e}")
    assert err < 2e-6
    assert np.array_equal(xd.cpu().numpy(), x.astype(np.complex64))
    sar.sar_fft_lines(n, 3, xd, xd, inverse)                     # in place
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), got)


@pytest.mark.parametrize("n", [100, 1000, 3000])
def test_lfm_spectrum_any_length(sar, orc, n):
    nc, tbp = n // 4, n / 8.0
    H = torch.empty(n, dtype=torch.complex64, device="cuda")
    sar.sar_make_lfm_spectrum(n, nc, tbp, H)
    torch.cuda.synchronize()
    ref = orc.matched_filter(n, sarsim.lfm_chirp(nc, tbp))
    assert M.rel_l2(H.cpu().numpy(), ref) < 2e-6
