"""GPU: the device echo simulator against the host generator, and ragged
batches (strips of mixed sizes in one CUDA-graph launch) against the oracle."""
import os

import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    torch.cuda.set_device(0)
    return sar


@pytest.mark.parametrize("spec", [sarsim.scene_256(),
                                  sarsim.SceneSpec(300, 512, [(10, 500), (150, 256), (299, 3)], (128, 64.0),
                                                   (64, 8.0), 10.0, 11),
                                  sarsim.SceneSpec(64, 1024, [(32, 512)], (1024, 512.0), (64, 16.0), None, 3)],
                         ids=["scene256", "wrapping", "noise_free"])
def test_device_simulator_matches_host_generator(sar, spec):
    host = sarsim.echo(spec)
    out = torch.empty((spec.n_az, spec.n_range), dtype=torch.complex64, device="cuda")
    sar.sar_simulate_echo(spec.n_az, spec.n_range, spec.targets, spec.range_chirp, spec.az_chirp, spec.snr_db,
                          spec.seed, out)
    dev = out.cpu().numpy()
    same = np.mean(dev == host)
    assert same > 0.999, same
    diff = np.abs(dev.astype(np.complex128) - host.astype(np.complex128))
    scale = np.maximum(np.abs(host.astype(np.complex128)), 1e-30)
    assert np.max(diff / scale) < 2.5e-7


def make_strips(sar, orc, shapes, seed=4):
    strips, keep, specs = [], [], []
    hr, ha = {}, {}
    for i, (n_range, n_az) in enumerate(shapes):
        spec = sarsim.strip_spec(seed * 100 + i, n_range, n_az, 1 + i % 4)
        raw = sarsim.echo(spec)
        L = spec.l_az if spec.l_az >= 256 else 256
        spec.l_az = L
        if n_range not in hr:
            hr[n_range] = torch.from_numpy(
                orc.matched_filter(n_range, sarsim.lfm_chirp(*spec.range_chirp)).astype(np.complex64)).cuda()
        if L not in ha:
            ha[L] = torch.from_numpy(orc.matched_filter(L, sarsim.lfm_chirp(*spec.az_chirp)).astype(np.complex64)).cuda()
        raw_d = torch.from_numpy(raw).cuda()
        img_d = torch.empty((n_range, n_az), dtype=torch.complex64, device="cuda")
        strips.append(dict(n_range=n_range, n_az=n_az, raw=raw_d, image=img_d, range_spectrum=hr[n_range],
                           az_spectrum=ha[L]))
        keep.append((raw, raw_d, img_d))
        specs.append(spec)
    return strips, keep, specs, hr, ha


def test_ragged_batch_vs_oracle(sar):
    orc = oracle.default()
    shapes = [(1024, 300), (256, 256), (4096, 777), (1024, 1000), (2048, 129), (256, 1), (512, 4096), (1024, 300)]
    strips, keep, specs, hr, ha = make_strips(sar, orc, shapes)
    batch = sar.sar_batch_create(strips)
    info = sar.sar_batch_info(batch)
    assert info["strips"] == len(shapes)
    assert info["samples"] == sum(a * b for a, b in shapes)
    assert info["range_classes"] == 5 and info["azimuth_classes"] == 4
    assert info["kernels_per_run"] == 1          # one persistent launch
    sar.sar_batch_run(batch)
    sar.sar_sync()
    sar.sar_batch_status(batch)
    for (raw, raw_d, img_d), spec, st in zip(keep, specs, strips):
        img = img_d.cpu().numpy()
        assert np.array_equal(raw_d.cpu().numpy(), raw)            # raw is read only
        Hr = hr[spec.n_range].cpu().numpy().astype(np.complex128)
        Ha = ha[spec.l_az].cpu().numpy().astype(np.complex128)
        ref = orc.rda(raw, Hr, Ha, l_az=spec.l_az, nthreads=NTHREADS)
        assert M.rel_l2(img, ref) < 2e-5, (spec.n_range, spec.n_az)
        for (a0, r0) in spec.targets:
            if spec.n_az >= 64:
                assert M.peak(img, (r0, a0)) == M.peak(ref, (r0, a0))
    # a second run of the same graph gives the same images
    first = [k[2].clone() for k in keep]
    sar.sar_batch_run(batch)
    sar.sar_sync()
    for a, k in zip(first, keep):
        assert torch.equal(a, k[2])
    batch.destroy()


def test_ragged_batch_long_range_lines_vs_oracle(sar):
    """Strips with range lines of 8192 and 16384 samples (one and two lines
    per work item, the engines with the most registers per thread) beside
    short ones, ragged azimuth counts, against the oracle."""
    orc = oracle.default()
    shapes = [(16384, 300), (8192, 517), (1024, 64), (16384, 129), (4096, 256), (8192, 40)]
    strips, keep, specs, hr, ha = make_strips(sar, orc, shapes, seed=7)
    batch = sar.sar_batch_create(strips)
    assert sar.sar_batch_info(batch)["kernels_per_run"] == 1
    sar.sar_batch_run(batch)
    sar.sar_batch_status(batch)
    for (raw, raw_d, img_d), spec in zip(keep, specs):
        img = img_d.cpu().numpy()
        Hr = hr[spec.n_range].cpu().numpy().astype(np.complex128)
        Ha = ha[spec.l_az].cpu().numpy().astype(np.complex128)
        ref = orc.rda(raw, Hr, Ha, l_az=spec.l_az, nthreads=NTHREADS)
        assert M.rel_l2(img, ref) < 2e-5, (spec.n_range, spec.n_az)
        for (a0, r0) in spec.targets:
            if spec.n_az >= 64:
                assert M.peak(img, (r0, a0)) == M.peak(ref, (r0, a0))
    batch.destroy()


def test_one_launch_equals_multi_kernel_graph(sar):
    """The one persistent kernel and the multi-kernel graph run the same line
    engines (same geometry, twiddles and filter order per length) and the
    corner turn is a copy either way: the images are bit-identical."""
    orc = oracle.default()
    shapes = [(1024, 300), (256, 256), (4096, 777), (2048, 129), (512, 4096), (8192, 100), (16384, 33)]
    strips, keep, specs, hr, ha = make_strips(sar, orc, shapes, seed=8)
    one = sar.sar_batch_create(strips)
    multi = sar.sar_batch_create(strips, flags=sar.SAR_BATCH_MULTI_KERNEL)
    assert sar.sar_batch_info(one)["kernels_per_run"] == 1
    assert sar.sar_batch_info(multi)["kernels_per_run"] > 1
    sar.sar_batch_run(one)
    sar.sar_batch_status(one)
    first = [k[2].clone() for k in keep]
    sar.sar_batch_run(multi)
    sar.sar_sync()
    for a, k, spec in zip(first, keep, specs):
        assert torch.equal(a, k[2]), (spec.n_range, spec.n_az)
    one.destroy()
    multi.destroy()


def test_ragged_batch_wait_timeout_is_reported(sar):
    """A strip whose completion counter can never reach its target
    (host-side injection: one range line more expected than it has) makes the
    azimuth items' bounded wait run out: sar_batch_status reports
    SAR_ERR_TIMEOUT within the bound, the record is cleared, the context stays
    usable and a batch created without the injection computes normally."""
    orc = oracle.default()
    shapes = [(1024, 300), (2048, 129), (4096, 64)]
    strips, keep, specs, hr, ha = make_strips(sar, orc, shapes, seed=9)
    os.environ["SAR_FAULT_INJECT_BATCH_WAIT"] = "1"
    os.environ["SAR_WAIT_CYCLES"] = "20000000"          # about ten milliseconds
    try:
        bad = sar.sar_batch_create(strips)
    finally:
        del os.environ["SAR_FAULT_INJECT_BATCH_WAIT"]
        del os.environ["SAR_WAIT_CYCLES"]
    import time
    t0 = time.perf_counter()
    sar.sar_batch_run(bad)
    with pytest.raises(sar.SarError) as e:
        sar.sar_batch_status(bad)
    assert e.value.status == sar.SAR_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    sar.sar_batch_status(bad)                            # the record was cleared
    bad.destroy()
    good = sar.sar_batch_create(strips)
    sar.sar_batch_run(good)
    sar.sar_batch_status(good)
    for (raw, raw_d, img_d), spec in zip(keep, specs):
        Hr = hr[spec.n_range].cpu().numpy().astype(np.complex128)
        Ha = ha[spec.l_az].cpu().numpy().astype(np.complex128)
        ref = orc.rda(raw, Hr, Ha, l_az=spec.l_az, nthreads=NTHREADS)
        assert M.rel_l2(img_d.cpu().numpy(), ref) < 2e-5
    good.destroy()


def test_batch_refuses_bad_strips(sar):
    x = torch.empty(1024, dtype=torch.complex64, device="cuda")
    bad = [dict(n_range=1000, n_az=4, raw=x, image=x, range_spectrum=x, az_spectrum=x)]
    with pytest.raises(sar.SarError) as e:
        sar.sar_batch_create(bad)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    bad = [dict(n_range=256, n_az=20000, raw=x, image=x, range_spectrum=x, az_spectrum=x)]
    with pytest.raises(sar.SarError):
        sar.sar_batch_create(bad)
    with pytest.raises(sar.SarError):
        sar.sar_batch_create([dict(n_range=256, n_az=4, raw=np.zeros(4, np.complex64), image=x,
                                   range_spectrum=x, az_spectrum=x)])


def test_ragged_batch_exact_azimuth_vs_oracle(sar):
    """SAR_BATCH_EXACT_AZIMUTH: every strip's azimuth lines compressed at
    exactly n_az (the oracle's circular correlation at that length; no zero
    padding), with azimuth spectra of n_az values."""
    orc = oracle.default()
    shapes = [(1024, 300), (256, 256), (2048, 777), (1024, 1000), (512, 129), (256, 77), (1024, 300), (512, 128)]
    strips, keep, specs, refs = [], [], [], []
    hr, ha = {}, {}
    for i, (n_range, n_az) in enumerate(shapes):
        (ncr, tbr), _ = sarsim.scaled_chirps(n_range, 256)
        nca = max(4, n_az // 4)
        tba = max(1.0, nca / 8.0)
        targets = [(n_az // 2, n_range // 2)]
        spec = sarsim.SceneSpec(n_az=n_az, n_range=n_range, targets=targets, range_chirp=(ncr, tbr),
                                az_chirp=(nca, tba), snr_db=20.0, seed=60 + i)
        raw = sarsim.echo(spec)
        if n_range not in hr:
            hr[n_range] = orc.matched_filter(n_range, sarsim.lfm_chirp(ncr, tbr))
        key = (n_az, nca)
        if key not in ha:
            ha[key] = orc.matched_filter(n_az, sarsim.lfm_chirp(nca, tba))
        raw_d = torch.from_numpy(raw).cuda()
        img_d = torch.empty((n_range, n_az), dtype=torch.complex64, device="cuda")
        strips.append(dict(n_range=n_range, n_az=n_az, raw=raw_d, image=img_d,
                           range_spectrum=torch.from_numpy(hr[n_range].astype(np.complex64)).cuda(),
                           az_spectrum=torch.from_numpy(ha[key].astype(np.complex64)).cuda()))
        keep.append((raw, raw_d, img_d, strips[-1]))
        specs.append(spec)
        refs.append(orc.rda(raw, hr[n_range].astype(np.complex64).astype(np.complex128),
                            ha[key].astype(np.complex64).astype(np.complex128), nthreads=NTHREADS))
    batch = sar.sar_batch_create(strips, flags=sar.SAR_BATCH_EXACT_AZIMUTH)
    info = sar.sar_batch_info(batch)
    assert info["strips"] == len(shapes)
    sar.sar_batch_run(batch)
    sar.sar_sync()
    for (raw, raw_d, img_d, _), spec, ref in zip(keep, specs, refs):
        img = img_d.cpu().numpy()
        assert np.array_equal(raw_d.cpu().numpy(), raw)
        err = M.rel_l2(img, ref)
        print(f"\nEXACT {spec.n_range}x{spec.n_az}: rel_l2 {err:.2e}")
        assert err < 2e-5, (spec.n_range, spec.n_az)
        (a0, r0), = spec.targets
        assert M.peak(img, (r0, a0)) == M.peak(ref, (r0, a0)) == (r0, a0)
    batch.destroy()
    x = torch.empty(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(sar.SarError) as e:
        sar.sar_batch_create([dict(n_range=256, n_az=9000, raw=x, image=x, range_spectrum=x, az_spectrum=x)],
                             flags=sar.SAR_BATCH_EXACT_AZIMUTH)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED


def test_multi_kernel_graph_autotuned_vs_oracle(sar):
    """SAR_BATCH_AUTOTUNE times every schedule of each class's length at batch
    creation and gives the class the fastest with a segment-table kernel; the
    images still match the oracle.  Refused for the one-launch kernel."""
    orc = oracle.default()
    shapes = [(1024, 200), (2048, 129), (512, 256), (1024, 77)]
    strips, keep, specs, hr, ha = make_strips(sar, orc, shapes, seed=12)
    with pytest.raises(sar.SarError) as e:
        sar.sar_batch_create(strips, flags=sar.SAR_BATCH_AUTOTUNE)
    assert e.value.status == sar.SAR_ERR_INVALID_ARG
    batch = sar.sar_batch_create(strips, flags=sar.SAR_BATCH_MULTI_KERNEL | sar.SAR_BATCH_AUTOTUNE)
    try:
        assert sar.sar_batch_info(batch)["kernels_per_run"] > 1
        sar.sar_batch_run(batch)
        sar.sar_sync()
        for (raw, raw_d, img_d), spec in zip(keep, specs):
            Hr = hr[spec.n_range].cpu().numpy().astype(np.complex128)
            Ha = ha[spec.l_az].cpu().numpy().astype(np.complex128)
            ref = orc.rda(raw, Hr, Ha, l_az=spec.l_az, nthreads=NTHREADS)
            assert M.rel_l2(img_d.cpu().numpy(), ref) < 2e-5, (spec.n_range, spec.n_az)
    finally:
        batch.destroy()
        # the tuning made its winners the preferred schedules: back to the
        # compiled defaults (the first schedule of each length)
        for n in (256, 512, 1024, 2048):
            sar.sar_set_preferred_schedule(sar.schedules(n)[0]["name"])
