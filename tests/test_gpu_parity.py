"""GPU parity: every entry point of the C-ABI against the FP64 oracle.

Tolerances (relative L2 over the compared array, FP64):
* one FP32 FFT of length N <= 16384: 2e-6 -- FP32 unit roundoff 6e-8 times
  an error growth of order log2 N for a Cooley-Tukey transform with accurate
  twiddles, with margin;
* one fused line compression (two transforms + multiply): 4e-6;
* a whole image (three passes): 2e-5, the acceptance bound for images, with
  compressed peaks at exactly the planted positions and PSLR / ISLR / SNR
  within 0.05 dB of the oracle's;
* the corner turn is a copy: bit-exact.
"""
import os

import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NS = [256, 512, 1024, 2048, 4096, 8192, 16384]
NTHREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar   # must load: no fallback on a GPU machine
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    torch.cuda.set_device(0)
    return sar


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rand_c64(count, seed, stream=7):
    return sarsim.complex_gaussian(seed, stream, count, 1.0)


def empty_c64(*shape):
    return torch.empty(shape, dtype=torch.complex64, device="cuda")


# ---------------------------------------------------------------------------
# the line FFT engine on its own
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_fft_lines_vs_oracle(sar, orc, n, inverse):
    n_lines = 37 if n <= 4096 else 5          # not a multiple of the lines per block
    x = rand_c64(n_lines * n, seed=n).reshape(n_lines, n)
    y = empty_c64(n_lines, n)
    sar.sar_fft_lines(n, n_lines, dev(x), y, inverse)
    got = host(y)
    for l in range(n_lines):
        ref = orc.fft(x[l], inverse=inverse)
        assert M.rel_l2(got[l], ref) < 2e-6, (n, l)


@pytest.mark.parametrize("n", [256, 4096, 16384])
def test_fft_in_place_equals_out_of_place(sar, n):
    x = dev(rand_c64(3 * n, seed=5).reshape(3, n))
    y = empty_c64(3, n)
    sar.sar_fft_lines(n, 3, x, y)
    sar.sar_fft_lines(n, 3, x, x)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("n,nc,tbp", [(256, 64, 32.0), (256, 64, 16.0), (4096, 512, 256.0),
                                      (4096, 1024, 128.0), (16384, 2048, 1024.0), (1024, 1024, 512.0)])
def test_lfm_spectrum_vs_oracle(sar, orc, n, nc, tbp):
    out = empty_c64(n)
    sar.sar_make_lfm_spectrum(n, nc, tbp, out)
    ref = orc.matched_filter(n, sarsim.lfm_chirp(nc, tbp))
    assert M.rel_l2(host(out), ref) < 2e-6


# ---------------------------------------------------------------------------
# the fused passes
# ---------------------------------------------------------------------------

def make_plan(sar, n_range, n_az, Hr, Ha):
    return sar.sar_plan_create(n_range, n_az, dev(Hr.astype(np.complex64)), dev(Ha.astype(np.complex64)))


@pytest.mark.parametrize("n", NS)
def test_range_compress_vs_oracle(sar, orc, n):
    n_az = 256
    Hr = orc.matched_filter(n, sarsim.lfm_chirp(n // 8, n / 16)).astype(np.complex64)
    Ha = rand_c64(n_az, seed=3)
    plan = make_plan(sar, n, n_az, Hr, Ha)
    x = rand_c64(n_az * n, seed=11 + n).reshape(n_az, n)
    xd = dev(x)
    out = empty_c64(n_az, n)
    sar.sar_range_compress_oop(plan, xd, out)      # out of place: input untouched
    sar.sar_range_compress(plan, xd)               # in place
    got = host(xd)
    assert np.array_equal(host(out), got)
    ref = orc.compress_lines(x, Hr.astype(np.complex128), nthreads=NTHREADS)
    assert M.rel_l2(got, ref) < 4e-6
    plan.destroy()


@pytest.mark.parametrize("n", NS)
def test_azimuth_compress_vs_oracle(sar, orc, n):
    Ha = rand_c64(n, seed=21 + n)                     # an arbitrary spectrum, not a chirp
    Hr = rand_c64(256, seed=4)
    plan = make_plan(sar, 256, n, Hr, Ha)
    x = rand_c64(256 * n, seed=31 + n).reshape(256, n)
    xd = dev(x)
    sar.sar_azimuth_compress(plan, xd)
    got = host(xd)
    ref = orc.compress_lines(x, Ha.astype(np.complex128), nthreads=NTHREADS)
    assert M.rel_l2(got, ref) < 4e-6
    plan.destroy()


def _all_schedules():
    import ctypes
    import importlib
    try:
        sar = importlib.import_module("paper_2604_03585_gb300")
    except ImportError:
        return []
    return [sar.sar_schedule_get(i)["name"] for i in range(sar.sar_schedule_count())]


@pytest.mark.parametrize("name", _all_schedules() or ["n4096_e64_r64x64_l1"])
def test_every_schedule_vs_oracle(sar, orc, name):
    d = [x for x in sar.schedules() if x["name"] == name][0]
    n, n_az = d["n"], 256
    Hr = rand_c64(n, seed=77 + n)
    Ha = rand_c64(n_az, seed=78)
    plan = sar.sar_plan_create_ex(n, n_az, dev(Hr), dev(Ha), range_schedule=name)
    assert sar.sar_plan_get_schedules(plan)[0]["name"] == name
    n_lines = n_az
    x = rand_c64(n_lines * n, seed=79 + n).reshape(n_lines, n)
    xd = dev(x)
    sar.sar_range_compress(plan, xd)
    got = host(xd)
    ref = orc.compress_lines(x, Hr.astype(np.complex128), nthreads=NTHREADS)
    assert M.rel_l2(got, ref) < 4e-6
    plan.destroy()


def _persistent_schedules():
    return [n for n in _all_schedules() if n.endswith("_p")]


@pytest.mark.parametrize("name", _persistent_schedules() or ["n4096_e32_r16x16x16_p"])
def test_persistent_many_lines_per_block(sar, orc, name):
    """More lines than resident blocks: every block loops, double-buffering
    its TMA copies; in place and out of place."""
    d = [x for x in sar.schedules() if x["name"] == name][0]
    n = d["n"]
    n_lines = 4096 if n <= 4096 else 2048
    Hr = rand_c64(n, seed=91 + n)
    Ha = rand_c64(n_lines, seed=92)
    plan = sar.sar_plan_create_ex(n, n_lines, dev(Hr), dev(Ha), range_schedule=name)
    x = rand_c64(n_lines * n, seed=93 + n).reshape(n_lines, n)
    xd = dev(x)
    out = empty_c64(n_lines, n)
    sar.sar_range_compress_oop(plan, xd, out)
    sar.sar_range_compress(plan, xd)
    sar.sar_plan_status(plan)
    got = host(out)
    assert np.array_equal(host(xd), got)
    ref = orc.compress_lines(x, Hr.astype(np.complex128), nthreads=NTHREADS)
    assert M.rel_l2(got, ref) < 4e-6
    plan.destroy()


def test_persistent_wait_timeout_is_reported(sar):
    """A copy that is never started (host-side injection) makes the bounded
    device wait run out: the plan reports SAR_ERR_TIMEOUT, the context stays
    usable and the next plan computes normally."""
    n, n_lines = 4096, 1024
    name = "n4096_e32_r16x16x16_p"
    Hr, Ha = rand_c64(n, 1), rand_c64(n_lines, 2)
    os.environ["SAR_FAULT_INJECT_SKIP_LINE"] = "700"
    os.environ["SAR_WAIT_CYCLES"] = "2000000"          # about a millisecond
    try:
        plan = sar.sar_plan_create_ex(n, n_lines, dev(Hr), dev(Ha), range_schedule=name)
    finally:
        del os.environ["SAR_FAULT_INJECT_SKIP_LINE"]
        del os.environ["SAR_WAIT_CYCLES"]
    x = dev(rand_c64(n_lines * n, seed=5).reshape(n_lines, n))
    sar.sar_range_compress(plan, x)
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_status(plan)
    assert e.value.status == sar.SAR_ERR_TIMEOUT
    sar.sar_plan_status(plan)                           # the record was cleared
    plan.destroy()
    plan = sar.sar_plan_create_ex(n, n_lines, dev(Hr), dev(Ha), range_schedule=name)
    y = empty_c64(n_lines, n)
    sar.sar_range_compress_oop(plan, x, y)
    sar.sar_plan_status(plan)
    sar.sar_sync()
    plan.destroy()


def _ct_schedules():
    try:
        import paper_2604_03585_gb300 as sar
    except ImportError:
        return []
    out = []
    for name in _all_schedules():
        d = [x for x in sar.schedules() if x["name"] == name][0]
        out.append(name)
    return out


@pytest.mark.parametrize("name", [n for n in _all_schedules()] or ["n4096_e32_r16x16x16_sr1"])
def test_folded_corner_turn_matches_unfolded(sar, orc, name):
    """sar_rda_process with the corner turn folded into the range pass gives
    bit-for-bit the result of the three separate kernels (same schedule), and
    both match the oracle; raw is left untouched by the folded path."""
    d = [x for x in sar.schedules() if x["name"] == name][0]
    n_range = d["n"]
    n_az = 256
    Hr, Ha = rand_c64(n_range, seed=5 + n_range), rand_c64(n_az, seed=6)
    raw = rand_c64(n_az * n_range, seed=7 + n_range).reshape(n_az, n_range)
    folded = sar.sar_plan_create_ex(n_range, n_az, dev(Hr), dev(Ha), range_schedule=name)
    if not sar.sar_plan_folds_corner_turn(folded):
        folded.destroy()
        pytest.skip("schedule has no folded corner turn")
    plain = sar.sar_plan_create_ex(n_range, n_az, dev(Hr), dev(Ha), range_schedule=name,
                                   flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
    assert not sar.sar_plan_folds_corner_turn(plain)
    r1, r2 = dev(raw), dev(raw)
    i1, i2 = empty_c64(n_range, n_az), empty_c64(n_range, n_az)
    sar.sar_rda_process(folded, r1, i1)
    sar.sar_rda_process(plain, r2, i2)
    a, b = host(i1), host(i2)
    assert np.array_equal(a, b)
    assert np.array_equal(host(r1), raw)
    ref = orc.rda(raw, Hr.astype(np.complex128), Ha.astype(np.complex128), nthreads=NTHREADS)
    assert M.rel_l2(a, ref) < 1e-5
    folded.destroy()
    plain.destroy()


@pytest.mark.parametrize("n_range,n_az", [(4096, 36), (2048, 100), (8192, 12), (4096, 300), (2048, 260)])
def test_folded_corner_turn_at_narrow_images(sar, n_range, n_az):
    """The default folded range pass writes its image tiles as tensor-store
    boxes of 4 azimuth samples; image rows of n_az = 4 (mod 8) samples put
    every other box at a 16-byte (not 32-byte) offset, and widths that are
    not powers of two run the mixed-radix or zero-padded azimuth pass.  The
    image equals the unfolded path's with the same range schedule (the
    default fold's) bit for bit."""
    Hr, Ha = rand_c64(n_range, seed=11 + n_az), rand_c64(n_az, seed=12)
    raw = rand_c64(n_az * n_range, seed=13 + n_range).reshape(n_az, n_range)
    folded = sar.sar_plan_create(n_range, n_az, dev(Hr), dev(Ha))
    name = sar.sar_plan_get_schedules(folded)[0]["name"]
    plain = sar.sar_plan_create_ex(n_range, n_az, dev(Hr), dev(Ha), range_schedule=name,
                                   flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
    assert sar.sar_plan_folds_corner_turn(folded) and not sar.sar_plan_folds_corner_turn(plain)
    i1, i2 = empty_c64(n_range, n_az), empty_c64(n_range, n_az)
    sar.sar_rda_process(folded, dev(raw), i1)
    sar.sar_rda_process(plain, dev(raw), i2)
    assert np.array_equal(host(i1), host(i2))
    folded.destroy()
    plain.destroy()


def test_autotune_picks_a_valid_schedule(sar):
    best, ms, allt = sar.sar_autotune(1024, 2048, reps=3)
    assert best["n"] == 1024 and ms > 0
    assert set(allt) == {d["name"] for d in sar.schedules(1024)}
    assert min(allt.values()) == pytest.approx(ms)
    best_ct, ms_ct, all_ct = sar.sar_autotune(4096, 256, reps=2, kind=sar.SAR_TUNE_RANGE_CT)
    assert best_ct["name"] in all_ct and ms_ct == pytest.approx(min(all_ct.values()))
    plan = sar.sar_plan_create(4096, 256, empty_c64(4096), empty_c64(256))
    assert sar.sar_plan_folds_corner_turn(plan)
    assert sar.sar_plan_get_schedules(plan)[0]["name"] == best_ct["name"]
    plan.destroy()
    with pytest.raises(sar.SarError):
        sar.sar_plan_create_ex(1024, 256, empty_c64(1024), empty_c64(256), range_schedule="n4096_e64_r64x64_l1")


# ---------------------------------------------------------------------------
# the corner turn: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 7), (7, 1), (33, 65), (17, 130), (1000, 3),
                                       (256, 256), (4096, 4096), (512, 16384), (3000, 1001)])
def test_transpose_bit_exact(sar, rows, cols):
    x = torch.randn(rows, cols, dtype=torch.complex64, device="cuda")
    y = empty_c64(cols, rows)
    sar.sar_transpose(rows, cols, x, y)
    torch.cuda.synchronize()
    assert torch.equal(y, x.t().contiguous())


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("rows,cols", [(4096, 4096), (128, 64), (192, 320), (100, 64), (64, 1000)])
def test_transpose_variants_bit_exact(sar, variant, rows, cols):
    """Both corner-turn kernels (32 x 32 tiles of 8-byte accesses; 64 x 64
    tiles of 16-byte accesses where rows and columns are multiples of 64,
    the 32 x 32 kernel otherwise) move every sample exactly."""
    x = torch.randn(rows, cols, dtype=torch.complex64, device="cuda")
    y = empty_c64(cols, rows)
    sar.sar_set_corner_turn_variant(variant)
    try:
        sar.sar_transpose(rows, cols, x, y)
        torch.cuda.synchronize()
    finally:
        sar.sar_set_corner_turn_variant(0)
    assert torch.equal(y, x.t().contiguous())


def test_corner_turn_plan_shape(sar):
    n_az, n_r = 512, 2048
    plan = make_plan(sar, n_r, n_az, rand_c64(n_r, 1), rand_c64(n_az, 2))
    x = torch.randn(n_az, n_r, dtype=torch.complex64, device="cuda")
    y = empty_c64(n_r, n_az)
    sar.sar_corner_turn(plan, x, y)
    torch.cuda.synchronize()
    assert torch.equal(y, x.t().contiguous())
    plan.destroy()


# ---------------------------------------------------------------------------
# whole scenes
# ---------------------------------------------------------------------------

def gpu_filters(sar, spec):
    Hr = empty_c64(spec.n_range)
    Ha = empty_c64(spec.az_len)
    sar.sar_make_lfm_spectrum(spec.n_range, *spec.range_chirp, Hr)
    sar.sar_make_lfm_spectrum(spec.az_len, *spec.az_chirp, Ha)
    return Hr, Ha


def oracle_filters(orc, spec):
    return (orc.matched_filter(spec.n_range, sarsim.lfm_chirp(*spec.range_chirp)),
            orc.matched_filter(spec.az_len, sarsim.lfm_chirp(*spec.az_chirp)))


def check_image(img, ref, spec, quality=True):
    assert img.shape == ref.shape == (spec.n_range, spec.n_az)
    err = M.rel_l2(img, ref)
    assert err <= 2e-5, err
    tg = [(r0, a0) for (a0, r0) in spec.targets]
    for t in tg:
        assert M.peak(img, t) == t
        assert M.peak(ref, t) == t
    if quality:
        qg, qr = M.quality(img, tg), M.quality(ref, tg)
        for a, b in zip(qg["targets"], qr["targets"]):
            assert a["pos"] == b["pos"]
            for k in ("pslr_axis0", "pslr_axis1", "islr_axis0", "islr_axis1", "snr"):
                assert abs(a[k] - b[k]) <= 0.05, (k, a[k], b[k])
    return err


def run_scene(sar, spec, Hr, Ha):
    raw = sarsim.echo(spec)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha)
    raw_d = dev(raw)
    img_d = empty_c64(spec.n_range, spec.n_az)
    sar.sar_rda_process(plan, raw_d, img_d)
    img = host(img_d)
    plan.destroy()
    return raw, img


def test_scene_256_gpu_filters(sar, orc):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    raw, img = run_scene(sar, spec, Hr, Ha)
    ref = orc.rda(raw, *oracle_filters(orc, spec))
    check_image(img, ref, spec)


def test_scene_256_shared_filters(sar, orc):
    """Same complex64 filter spectra on both sides: isolates the compressor."""
    spec = sarsim.scene_256()
    Hr, Ha = (h.astype(np.complex64) for h in oracle_filters(orc, spec))
    raw, img = run_scene(sar, spec, dev(Hr), dev(Ha))
    ref = orc.rda(raw, Hr.astype(np.complex128), Ha.astype(np.complex128))
    err = check_image(img, ref, spec)
    assert err < 5e-6


def test_scene_4096_full_size(sar, orc):
    """The 4096 x 4096 workload in the benchmark's launch configuration,
    compared with the oracle on every sample."""
    spec = sarsim.scene_4096()
    Hr, Ha = gpu_filters(sar, spec)
    raw, img = run_scene(sar, spec, Hr, Ha)
    ref = orc.rda(raw, *oracle_filters(orc, spec), nthreads=NTHREADS)
    check_image(img, ref, spec)


@pytest.mark.parametrize("n_az,n_range", [(512, 2048), (2048, 512), (16384, 256), (256, 16384)])
def test_non_square_scenes(sar, orc, n_az, n_range):
    rc, ac = sarsim.scaled_chirps(n_range, n_az)
    tg = sarsim.place_targets(9, n_az, n_range, 3, margin_az=min(64, n_az // 8),
                              margin_r=min(64, n_range // 8), min_sep=16)
    spec = sarsim.SceneSpec(n_az, n_range, tg, rc, ac, 10.0, 9)
    Hr, Ha = gpu_filters(sar, spec)
    raw, img = run_scene(sar, spec, Hr, Ha)
    ref = orc.rda(raw, *oracle_filters(orc, spec), nthreads=NTHREADS)
    check_image(img, ref, spec, quality=False)


@pytest.mark.parametrize("make", [sarsim.scene_256, sarsim.scene_4096], ids=["256", "4096"])
def test_unfused_pipeline_matches_fused_and_oracle(sar, orc, make):
    """The unfused comparison pipeline (FFT kernel, multiply kernel, IFFT
    kernel per pass) computes the same image as the fused kernels."""
    spec = make()
    Hr, Ha = gpu_filters(sar, spec)
    raw, fused = run_scene(sar, spec, Hr, Ha)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha)
    raw_d = dev(raw)
    img_d = empty_c64(spec.n_range, spec.n_az)
    sar.sar_rda_process_unfused(plan, raw_d, img_d)
    unf = host(img_d)
    plan.destroy()
    assert M.rel_l2(unf, fused) < 1e-5
    ref = orc.rda(raw, *oracle_filters(orc, spec), nthreads=NTHREADS)
    check_image(unf, ref, spec, quality=spec.n_az == 256)


def test_noise_free_peak_value(sar):
    spec = sarsim.scene_256()
    spec.snr_db = None
    Hr, Ha = gpu_filters(sar, spec)
    _, img = run_scene(sar, spec, Hr, Ha)
    assert abs(img[128, 128] - 64 * 64) < 1e-4 * 64 * 64


# ---------------------------------------------------------------------------
# properties of the product path
# ---------------------------------------------------------------------------

def test_deterministic(sar):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    _, a = run_scene(sar, spec, Hr, Ha)
    _, b = run_scene(sar, spec, Hr, Ha)
    assert np.array_equal(a, b)


def test_host_entry_point_matches_device(sar):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    raw, img = run_scene(sar, spec, Hr, Ha)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha)
    raw_h = torch.from_numpy(raw).pin_memory()
    img_h = torch.empty((spec.n_range, spec.n_az), dtype=torch.complex64).pin_memory()
    sar.sar_rda_process_host(plan, raw_h, img_h)
    assert np.array_equal(img_h.numpy(), img)
    assert np.array_equal(raw_h.numpy(), raw)        # host input untouched
    plan.destroy()


@pytest.mark.parametrize("flags", [0, 1], ids=["folded-pipelined", "unfolded"])
def test_host_entry_point_4096_matches_device(sar, flags):
    """The host-buffer call (chunked copy / compute pipeline on folded plans)
    gives bit for bit the device-buffer result on the 4096^2 scene."""
    spec = sarsim.scene_4096()
    raw = sarsim.echo(spec)
    Hr, Ha = gpu_filters(sar, spec)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha, flags=flags)
    img = empty_c64(spec.n_range, spec.n_az)
    sar.sar_rda_process_oop(plan, dev(raw), empty_c64(spec.n_az, spec.n_range), img)
    raw_h = torch.from_numpy(raw).pin_memory()
    img_h = torch.empty((spec.n_range, spec.n_az), dtype=torch.complex64).pin_memory()
    for _ in range(2):                                 # the second call reuses streams and events
        sar.sar_rda_process_host(plan, raw_h, img_h)
        assert np.array_equal(img_h.numpy(), host(img))
    assert np.array_equal(raw_h.numpy(), raw)
    plan.destroy()


@pytest.mark.parametrize("size,flags", [(256, 0), (4096, 0), (4096, 1)],
                         ids=["256-pipelined", "4096-pipelined", "4096-unfolded"])
def test_host_n_scenes_match_device(sar, size, flags):
    """sar_rda_process_host_n over three different scenes (two device staging
    sets on folded plans, the sets reused by the third scene) gives each
    scene's device-buffer image bit for bit, and a second call reuses the
    pipeline's streams and events."""
    import dataclasses
    base = sarsim.scene_256() if size == 256 else sarsim.scene_4096()
    specs = [dataclasses.replace(base, seed=base.seed + q) for q in range(3)]
    Hr, Ha = gpu_filters(sar, base)
    plan = sar.sar_plan_create(base.n_range, base.n_az, Hr, Ha, flags=flags)
    raws = [sarsim.echo(sp) for sp in specs]
    want = []
    for raw in raws:
        img = empty_c64(base.n_range, base.n_az)
        sar.sar_rda_process_oop(plan, dev(raw), empty_c64(base.n_az, base.n_range), img)
        want.append(host(img))
    assert not np.array_equal(want[0], want[1])
    raws_h = [torch.from_numpy(r).pin_memory() for r in raws]
    imgs_h = [torch.empty((base.n_range, base.n_az), dtype=torch.complex64).pin_memory() for _ in raws]
    for _ in range(2):
        for m in imgs_h:
            m.zero_()
        sar.sar_rda_process_host_n(plan, raws_h, imgs_h)
        for m, w in zip(imgs_h, want):
            assert np.array_equal(m.numpy(), w)
    for r, r_h in zip(raws, raws_h):
        assert np.array_equal(r_h.numpy(), r)            # host echoes untouched
    sar.sar_rda_process_host_n(plan, raws_h[:1], imgs_h[:1])   # one scene: the single-call pipeline
    assert np.array_equal(imgs_h[0].numpy(), want[0])
    assert sar.sar_plan_folds_corner_turn(plan) == (flags == 0)
    plan.destroy()


def test_host_n_refusals(sar):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha)
    raw_h = torch.zeros((spec.n_az, spec.n_range), dtype=torch.complex64).pin_memory()
    img_h = torch.empty((spec.n_range, spec.n_az), dtype=torch.complex64).pin_memory()
    sar.sar_rda_process_host_n(plan, [], [])                              # nothing to do
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_process_host_n(plan, [raw_h, 0], [img_h, img_h])      # a NULL echo
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        sar.sar_rda_process_host_n(plan, [raw_h], [img_h, img_h])
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_process_host_n(plan, [raw_h, raw_h], [img_h, raw_h])   # an image over an echo
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    sar.sar_rda_process_host_n(plan, [raw_h, raw_h, raw_h], [img_h, img_h, img_h])   # one image buffer, three scenes
    ref = torch.empty_like(img_h).pin_memory()
    sar.sar_rda_process_host(plan, raw_h, ref)
    assert torch.equal(img_h, ref)
    plan.destroy()


def test_guard_bands_untouched(sar):
    n_az, n_r, guard = 256, 512, 4096
    plan = make_plan(sar, n_r, n_az, rand_c64(n_r, 1), rand_c64(n_az, 2))
    canary = complex(1234.5, -987.25)
    buf = torch.full((2 * guard + n_az * n_r,), canary, dtype=torch.complex64, device="cuda")
    out = torch.full((2 * guard + n_az * n_r,), canary, dtype=torch.complex64, device="cuda")
    buf[guard:guard + n_az * n_r] = torch.randn(n_az * n_r, dtype=torch.complex64, device="cuda")
    sar.sar_rda_process(plan, buf[guard:], out[guard:])
    torch.cuda.synchronize()
    for b in (buf, out):
        assert bool((b[:guard] == canary).all()) and bool((b[guard + n_az * n_r:] == canary).all())
    plan.destroy()


def test_bad_arguments_are_refused(sar):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    plan = sar.sar_plan_create(256, 256, Hr, Ha)
    good = empty_c64(256, 256)
    other = empty_c64(256, 256)
    host_arr = np.zeros((256, 256), np.complex64)
    with pytest.raises(sar.SarError) as e:
        sar.sar_range_compress(plan, host_arr)             # host memory
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    flat = empty_c64(256 * 256 + 1)
    with pytest.raises(sar.SarError) as e:
        sar.sar_range_compress(plan, flat[1:])              # 8-byte, not 16-byte, aligned
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_process(plan, good, good)                # image overlaps raw
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(256, 256 * 33, Hr, Ha)          # not a power of two and above 8192
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(256, 262144, Hr, Ha)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    sar.sar_rda_process(plan, good, other)                   # still usable afterwards
    sar.sar_sync()
    plan.destroy()


def test_allocation_failure_is_reported(sar):
    spec = sarsim.scene_256()
    Hr, Ha = gpu_filters(sar, spec)
    os.environ["SAR_FAULT_INJECT_ALLOC"] = "1"
    try:
        with pytest.raises(sar.SarError) as e:
            sar.sar_plan_create(256, 256, Hr, Ha)
        assert e.value.status == sar.SAR_ERR_OUT_OF_MEMORY
    finally:
        del os.environ["SAR_FAULT_INJECT_ALLOC"]
    sar.sar_plan_create(256, 256, Hr, Ha).destroy()


def test_empty_inputs(sar):
    sar.sar_fft_lines(256, 0, 0, 0)        # zero lines: nothing to do, no pointer needed
    sar.sar_sync()


# ---------------------------------------------------------------------------
# split-precision tensor-core DFTs (precision comparison on the 4096^2 scene)
# ---------------------------------------------------------------------------

PREC_GATES = {"FP16X2": 2e-5, "BF16X3": 2e-5, "BF16X2": 2e-4}


@pytest.mark.parametrize("engine", [0, 2, 1], ids=["tcgen05_tmem_a", "tcgen05_smem_a", "mma_sync"])
@pytest.mark.parametrize("prec", ["FP16X2", "BF16X2", "BF16X3"])
@pytest.mark.parametrize("make", [sarsim.scene_256, sarsim.scene_4096], ids=["256", "4096"])
def test_split_precision_vs_oracle(sar, orc, prec, make, engine):
    """Error of each split-precision variant against the FP64 oracle, stated
    for the record (rel-L2, peaks, PSLR/ISLR/SNR deltas); FP16 hi/lo and
    BF16 hi/mid/lo meet the image gate, BF16 hi/lo is reported with its own
    (looser) bound.  Both engines: tcgen05.mma with TMEM accumulators (the
    default) and the warp-level mma.sync form."""
    spec = make()
    Hr, Ha = gpu_filters(sar, spec)
    raw = sarsim.echo(spec)
    code = getattr(sar, "SAR_PREC_" + prec)
    plan = sar.sar_plan_create(spec.n_range, spec.n_az, Hr, Ha, precision=code)
    assert not sar.sar_plan_folds_corner_turn(plan)
    raw_d = dev(raw)
    img_d = empty_c64(spec.n_range, spec.n_az)
    sar.sar_set_split_engine(engine)
    try:
        sar.sar_rda_process(plan, raw_d, img_d)
        sar.sar_plan_status(plan)
    finally:
        sar.sar_set_split_engine(0)
    img = host(img_d)
    plan.destroy()
    ref = orc.rda(raw, *oracle_filters(orc, spec), nthreads=NTHREADS)
    err = M.rel_l2(img, ref)
    tg = [(r0, a0) for (a0, r0) in spec.targets]
    qg, qr = M.quality(img, tg), M.quality(ref, tg)
    worst = {k: max(abs(a[k] - b[k]) for a, b in zip(qg["targets"], qr["targets"]))
             for k in ("pslr_axis0", "pslr_axis1", "islr_axis0", "islr_axis1", "snr")}
    print(f"\nPRECISION {prec} engine {engine} {spec.n_az}x{spec.n_range}: rel_l2={err:.3e} max_abs={M.max_abs(img, ref):.3e} "
          + " ".join(f"d_{k}={v:.4f}dB" for k, v in worst.items()))
    assert err <= PREC_GATES[prec], err
    for a, b in zip(qg["targets"], qr["targets"]):
        assert a["pos"] == b["pos"]
    if prec != "BF16X2":
        assert max(worst.values()) <= 0.05


def test_split_precision_refusals(sar):
    x = empty_c64(1024)
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(1024, 1024, x, x, precision=sar.SAR_PREC_FP16X2)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(1024, 1024, x, x, precision=9)
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    with pytest.raises(sar.SarError) as e:
        sar.sar_set_split_engine(3)
    assert e.value.status == sar.SAR_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# azimuth-major output: the fourth pass (transpose back)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_range,n_az,flags", [(4096, 4096, 0), (1024, 512, 1), (1000, 300, 0)],
                         ids=["4096-folded", "1024x512-unfolded", "1000x300-any-length"])
def test_azimuth_major_output(sar, n_range, n_az, flags):
    """SAR_PLAN_OUT_AZ_MAJOR returns exactly the transpose of the usual
    [n_range][n_az] image, from device and from host buffers."""
    Hr, Ha = rand_c64(n_range, seed=41), rand_c64(n_az, seed=42)
    raw = rand_c64(n_az * n_range, seed=43).reshape(n_az, n_range)
    ref_plan = sar.sar_plan_create(n_range, n_az, dev(Hr), dev(Ha), flags=flags)
    maj_plan = sar.sar_plan_create(n_range, n_az, dev(Hr), dev(Ha), flags=flags | sar.SAR_PLAN_OUT_AZ_MAJOR)
    r0, w0, img = dev(raw), empty_c64(n_az, n_range), empty_c64(n_range, n_az)
    sar.sar_rda_process_oop(ref_plan, r0, w0, img)
    r1, w1, out = dev(raw), empty_c64(n_az, n_range), empty_c64(n_az, n_range)
    sar.sar_rda_process_oop(maj_plan, r1, w1, out)
    ref = host(img)
    assert np.array_equal(host(out), ref.T)
    assert np.array_equal(host(r1), raw)
    out_h = torch.empty((n_az, n_range), dtype=torch.complex64).pin_memory()
    sar.sar_rda_process_host(maj_plan, torch.from_numpy(raw).pin_memory(), out_h)
    assert np.array_equal(out_h.numpy(), ref.T)
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_process(maj_plan, dev(raw), empty_c64(n_az, n_range))
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    ref_plan.destroy()
    maj_plan.destroy()


# ---------------------------------------------------------------------------
# twiddle tables against their FP64 closed form
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", NS + [32768, 65536, 131072])
def test_fft_of_impulse_is_the_closed_form_root(sar, n):
    """The FFT of the impulse at index 1 is exp(-2 pi i k / N) and of the one at
    N - 1 is exp(+2 pi i k / N): every output is a product of twiddle-table
    entries (FP64 phases rounded once to FP32, then the roots table of the
    cluster lengths), so each must equal the closed form to a few FP32 ulps;
    one wrong entry would show as an O(1) error."""
    x = np.zeros((2, n), np.complex64)
    x[0, 1] = 1.0
    x[1, n - 1] = 1.0
    xd = dev(x)
    out = torch.empty_like(xd)
    sar.sar_fft_lines(n, 2, xd, out)
    got = host(out).astype(np.complex128)
    k = np.arange(n)
    ref = np.stack([np.exp(-2j * np.pi * k / n), np.exp(2j * np.pi * k / n)])
    err = np.max(np.abs(got - ref))
    print(f"\nTWIDDLE n={n}: max |X - exp(-+2 pi i k/N)| = {err:.2e} ({err / 2 ** -24:.1f} x 2^-24)")
    assert err < 16 * 2 ** -24
