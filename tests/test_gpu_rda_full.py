"""GPU: the full Range-Doppler processor (azimuth FFT, RCMC, range-dependent
azimuth filter, IFFT) against the FP64 oracle written from Sec. IV-A."""
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


def run_full(sar, raw, Hr, geo, taps, unfolded=False):
    n_az, n_r = raw.shape
    Hr_d = torch.from_numpy(Hr.astype(np.complex64)).cuda()
    dummy = torch.zeros(n_az, dtype=torch.complex64, device="cuda")
    plan = sar.sar_plan_create(n_r, n_az, Hr_d, dummy, flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN if unfolded else 0)
    sar.sar_plan_set_geometry(plan, *geo.as_tuple(), taps)
    raw_d = torch.from_numpy(raw).cuda()
    work = torch.empty((n_r, n_az), dtype=torch.complex64, device="cuda")
    img = torch.empty((n_r, n_az), dtype=torch.complex64, device="cuda")
    sar.sar_rda_full(plan, raw_d, work, img)
    torch.cuda.synchronize()
    out = img.cpu().numpy()
    assert np.array_equal(raw_d.cpu().numpy(), raw)
    plan.destroy()
    return out


@pytest.mark.parametrize("taps", [16, 0])
@pytest.mark.parametrize("unfolded", [False, True], ids=["folded", "unfolded"])
def test_full_rda_small_vs_oracle(sar, taps, unfolded):
    orc = oracle.default()
    geo = sarsim.Geometry(10.0, 0.3, 4000.0)
    tg = [(500, 200), (300, 100), (700, 400)]
    raw = sarsim.echo_migration(1024, 512, tg, (64, 32.0), 512, geo, 20.0, 5)
    Hr = orc.matched_filter(512, sarsim.lfm_chirp(64, 32.0)).astype(np.complex64)
    img = run_full(sar, raw, Hr, geo, taps, unfolded)
    ref = orc.rda_full(raw, Hr.astype(np.complex128), geo, taps=taps, nthreads=NTHREADS)
    err = M.rel_l2(img, ref)
    assert err < 2e-5, err
    for (a0, n0) in tg:
        assert M.peak(img, (n0, a0)) == M.peak(ref, (n0, a0)) == (n0, a0)


def test_full_rda_4096_vs_oracle(sar):
    orc = oracle.default()
    tg, rc, ap, geo, snr, seed = sarsim.migration_scene_4096()
    raw = sarsim.echo_migration(4096, 4096, tg, rc, ap, geo, snr, seed)
    Hr = orc.matched_filter(4096, sarsim.lfm_chirp(*rc)).astype(np.complex64)
    img = run_full(sar, raw, Hr, geo, 16)
    ref = orc.rda_full(raw, Hr.astype(np.complex128), geo, taps=16, nthreads=NTHREADS)
    err = M.rel_l2(img, ref)
    print(f"\nFULL RDA 4096x4096: rel_l2 = {err:.3e}")
    assert err < 2e-5, err
    for (a0, n0) in tg:
        assert M.peak(img, (n0, a0)) == M.peak(ref, (n0, a0)) == (n0, a0)


@pytest.mark.parametrize("n_range,n_az,geo", [
    (512, 256, sarsim.Geometry(10.0, 0.3, 4000.0)),
    (1024, 4096, sarsim.Geometry(10.0, 0.3, 4000.0)),   # bins up to 5000: FP32 spacing 5e-4
    (4096, 512, sarsim.Geometry(2.0, 0.3, 100.0)),      # D down to 0.55: shifts up to ~3400 bins
    (256, 1024, sarsim.Geometry(5.0, 0.11, 37.3)),      # fractional r_near, kappa v_s = 0.55
    (300, 999, sarsim.Geometry(10.0, 0.3, 4000.0)),     # ragged in both: the last tiles partial
    (256, 512, sarsim.Geometry(3.0, 0.3, 2000.0)),      # ~200 rows per tile: the 128-bin tiles, staged
])
def test_rcmc_vs_oracle(sar, n_range, n_az, geo):
    """RCMC alone on white complex Gaussian range-Doppler data: every
    interpolation weight shows in the output, element by element.  The tiles
    stage their input rows in shared memory (up to ~200 rows per tile at
    256 x 512, kappa 3; a partial last tile in both directions at 300 x 999)
    or, where the migration is too wide for that, read global memory
    (256 x 1024 at kappa v_s 0.55, 4096 x 512 at kappa 2)."""
    orc = oracle.default()
    rd = sarsim.complex_gaussian(17, 0, n_range * n_az, 1.0).reshape(n_range, n_az)
    ref = orc.rcmc(rd, geo, taps=16)
    x = torch.from_numpy(rd).cuda()
    y = torch.empty_like(x)
    dummy = torch.zeros(max(n_range, n_az), dtype=torch.complex64, device="cuda")
    plan = sar.sar_plan_create(n_range, n_az, dummy[:n_range], dummy[:n_az])
    sar.sar_plan_set_geometry(plan, *geo.as_tuple(), 16)
    sar.sar_rcmc(plan, x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    plan.destroy()
    # FP32 weights on unit-variance data: ~16 taps x 1e-7 relative each
    err = np.abs(got - ref)
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    print(f"\nRCMC {n_range}x{n_az} kappa={geo.kappa} v_s={geo.v_s}: max {err.max() / scale:.2e} "
          f"rel_l2 {M.rel_l2(got, ref):.2e}")
    assert M.rel_l2(got, ref) < 2e-6
    assert err.max() < 2e-5 * scale


def test_geometry_refusals(sar):
    x = torch.zeros(256, dtype=torch.complex64, device="cuda")
    plan = sar.sar_plan_create(256, 256, x, x)
    with pytest.raises(sar.SarError):
        sar.sar_plan_set_geometry(plan, 1.0, 0.1, 100.0, 16)       # kappa * v_s <= 0.5
    with pytest.raises(sar.SarError):
        sar.sar_plan_set_geometry(plan, 10.0, 0.3, 100.0, 7)       # taps
    y = torch.empty((256, 256), dtype=torch.complex64, device="cuda")
    with pytest.raises(sar.SarError):
        sar.sar_rda_full(plan, y, torch.empty_like(y), torch.empty_like(y))   # no geometry yet
    with pytest.raises(sar.SarError):
        sar.sar_rcmc(plan, y, torch.empty_like(y))                           # no geometry yet
    sar.sar_plan_set_geometry(plan, 10.0, 0.3, 100.0, 0)
    with pytest.raises(sar.SarError):
        sar.sar_rcmc(plan, y, torch.empty_like(y))                           # taps = 0
    with pytest.raises(sar.SarError):
        sar.sar_rcmc(plan, y, y)                                             # overlap
    plan.destroy()


@pytest.mark.parametrize("n_az", [256, 512, 1024, 2048, 4096, 8192, 16384])
def test_full_rda_every_azimuth_length(sar, n_az):
    """The full processor at every azimuth length its kernels are compiled
    for (each with its own twiddle tables): one migrating target, 256 range
    bins, against the oracle."""
    orc = oracle.default()
    geo = sarsim.Geometry(10.0, 0.3, 4000.0)
    tg = [(n_az // 2, 128)]
    raw = sarsim.echo_migration(n_az, 256, tg, (32, 16.0), min(512, n_az // 2), geo, 20.0, 9)
    Hr = orc.matched_filter(256, sarsim.lfm_chirp(32, 16.0)).astype(np.complex64)
    img = run_full(sar, raw, Hr, geo, 16)
    ref = orc.rda_full(raw, Hr.astype(np.complex128), geo, taps=16, nthreads=NTHREADS)
    err = M.rel_l2(img, ref)
    print(f"\nFULL RDA n_az={n_az}: rel_l2 = {err:.3e}")
    assert err < 2e-5, err
    (a0, n0), = tg
    assert M.peak(img, (n0, a0)) == M.peak(ref, (n0, a0))
