"""GPU: lines longer than one thread block's shared memory (32768 ... 131072
samples), transformed by thread-block clusters through distributed shared
memory, against the FP64 oracle (the fused line compression of Sec. II-B and
the scene compression of Sec. IV-A at those lengths)."""
import os

import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = max(1, os.cpu_count() or 1)
LONG = [32768, 65536, 131072]
FFT_TOL = 2e-6      # one FP32 transform (as for the shorter lengths)
LINE_TOL = 4e-6     # one fused line: two transforms and the filter
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


def cluster_schedules(sar, n):
    return [d for d in sar.schedules(n) if d["cluster_blocks"] > 1]


def noise(seed, rows, n):
    return sarsim.complex_gaussian(seed, 0, rows * n, 1.0).reshape(rows, n)


def test_cluster_schedules_are_listed(sar):
    for n in LONG:
        ds = cluster_schedules(sar, n)
        assert ds, n
        for d in ds:
            assert d["n"] == n and d["n"] % d["cluster_blocks"] == 0
            assert d["threads_per_block"] * d["e"] * d["cluster_blocks"] == n


@pytest.mark.parametrize("n", LONG)
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_fft_long_lines_vs_oracle(sar, orc, n, inverse):
    x = noise(11, 3, n)
    ref = np.stack([orc.fft(row, inverse=inverse) for row in x])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    sar.sar_fft_lines(n, 3, xd, out, inverse)
    torch.cuda.synchronize()
    assert M.rel_l2(out.cpu().numpy(), ref) < FFT_TOL
    # in place as well
    sar.sar_fft_lines(n, 3, xd, xd, inverse)
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), out.cpu().numpy())


@pytest.mark.parametrize("n", LONG)
def test_lfm_spectrum_long(sar, orc, n):
    nc, tbp = n // 8, n / 16.0
    H = torch.empty(n, dtype=torch.complex64, device="cuda")
    sar.sar_make_lfm_spectrum(n, nc, tbp, H)
    torch.cuda.synchronize()
    ref = orc.matched_filter(n, sarsim.lfm_chirp(nc, tbp))
    assert M.rel_l2(H.cpu().numpy(), ref) < FFT_TOL


CLUSTER_SCHEDULES = [(n, f"n{n}_c{c}_m{m}_e32{v}") for (n, c, m) in
                     [(32768, 4, 8192), (32768, 2, 16384), (65536, 8, 8192), (65536, 4, 16384),
                      (131072, 8, 16384), (131072, 16, 8192)] for v in ("", "_sr")] + \
                    [(n, f"n{n}_c{c}_m{m}_e32{v}") for (n, c, m, v) in
                     [(32768, 8, 4096, "_sr"), (32768, 8, 4096, "_sr_b5"), (65536, 16, 4096, "_sr")]]


def test_cluster_schedule_list_is_complete(sar):
    assert sorted((n, d["name"]) for n in LONG for d in cluster_schedules(sar, n)) == sorted(CLUSTER_SCHEDULES)


@pytest.mark.parametrize("n,name", CLUSTER_SCHEDULES)
def test_fused_compression_every_cluster_schedule(sar, orc, n, name):
    """Range compression of 256 lines of n through each cluster schedule:
    y = IFFT(FFT(x) . H) per line (Sec. II-B), H of an LFM of n/8 samples."""
    n_az = 256
    x = noise(23, n_az, n)
    nc, tbp = n // 8, n / 16.0
    H = orc.matched_filter(n, sarsim.lfm_chirp(nc, tbp))
    Ha = orc.matched_filter(n_az, sarsim.lfm_chirp(64, 16.0))
    ref = orc.compress_lines(x, H, nthreads=NTHREADS)
    Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
    Had = torch.from_numpy(Ha.astype(np.complex64)).cuda()
    plan = sar.sar_plan_create_ex(n, n_az, Hd, Had, range_schedule=name)
    assert sar.sar_plan_get_schedules(plan)[0]["name"] == name
    assert not sar.sar_plan_folds_corner_turn(plan)
    xd = torch.from_numpy(x).cuda()
    sar.sar_range_compress(plan, xd)
    torch.cuda.synchronize()
    got = xd.cpu().numpy()
    plan.destroy()
    per_line = [M.rel_l2(got[i], ref[i]) for i in (0, 1, n_az // 2, n_az - 1)]
    print(f"\nLONG {name}: rel_l2 {M.rel_l2(got, ref):.2e}, worst sampled line {max(per_line):.2e}")
    assert M.rel_l2(got, ref) < LINE_TOL
    assert max(per_line) < LINE_TOL


@pytest.mark.parametrize("n_az,n_range", [(256, 32768), (32768, 256), (512, 65536)])
def test_scene_with_long_lines_vs_oracle(sar, orc, n_az, n_range):
    """The three-step scene compression (Sec. IV-A) with one dimension longer
    than a block's shared memory: point targets at their planted cells."""
    (ncr, tbr), (nca, tba) = sarsim.scaled_chirps(n_range, n_az)
    targets = [(n_az // 4, n_range // 3), (3 * n_az // 4, 2 * n_range // 3)]
    spec = sarsim.SceneSpec(n_az=n_az, n_range=n_range, targets=targets, range_chirp=(ncr, tbr),
                            az_chirp=(nca, tba), snr_db=20.0, seed=4)
    raw = sarsim.echo(spec)
    Hr = orc.matched_filter(n_range, sarsim.lfm_chirp(ncr, tbr))
    Ha = orc.matched_filter(n_az, sarsim.lfm_chirp(nca, tba))
    ref = orc.rda(raw, Hr, Ha, nthreads=NTHREADS)
    plan = sar.sar_plan_create(n_range, n_az, torch.from_numpy(Hr.astype(np.complex64)).cuda(),
                               torch.from_numpy(Ha.astype(np.complex64)).cuda())
    raw_d = torch.from_numpy(raw).cuda()
    img = torch.empty((n_range, n_az), dtype=torch.complex64, device="cuda")
    sar.sar_rda_process(plan, raw_d, img)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    plan.destroy()
    err = M.rel_l2(got, ref)
    print(f"\nLONG scene {n_az}x{n_range}: rel_l2 {err:.2e}")
    assert err < SCENE_TOL
    for (a0, r0) in targets:
        assert M.peak(got, (r0, a0)) == M.peak(ref, (r0, a0)) == (r0, a0)


def test_autotune_long(sar):
    best, best_ms, all_ms = sar.sar_autotune(32768, 384, reps=3)
    assert best["n"] == 32768 and best["cluster_blocks"] > 1
    assert best_ms > 0 and set(all_ms) == {d["name"] for d in cluster_schedules(sar, 32768)}
    sar.sar_set_preferred_schedule(best["name"])


def test_long_lines_refused_where_unsupported(sar):
    x = torch.zeros(32768, dtype=torch.complex64, device="cuda")
    with pytest.raises(sar.SarError) as e:
        sar.sar_fft_lines_static(32768, 1, x, x)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    a = torch.zeros(256, dtype=torch.complex64, device="cuda")
    plan = sar.sar_plan_create(256, 32768, a, x)
    sar.sar_plan_set_geometry(plan, 10.0, 0.3, 100.0, 16)
    img = torch.empty((256, 32768), dtype=torch.complex64, device="cuda")
    with pytest.raises(sar.SarError) as e:
        sar.sar_rda_full(plan, img, torch.empty_like(img), torch.empty_like(img))
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
    plan.destroy()
    with pytest.raises(sar.SarError) as e:
        sar.sar_plan_create(256, 262144, a, a)
    assert e.value.status == sar.SAR_ERR_UNSUPPORTED
