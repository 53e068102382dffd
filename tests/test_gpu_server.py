"""GPU: the continuous-batching request loop.  Every result is the same
alone and in the mix (bit for bit: same plan, same kernels), agrees with the
oracle, and the admission budget and timestamps behave."""
import numpy as np
import pytest

import oracle
import sarsim
from oracle import metrics as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    torch.cuda.set_device(0)
    return sar


@pytest.fixture(scope="module")
def classes(sar):
    orc = oracle.default()
    out = []
    for n in (256, 512, 1024):
        spec = sarsim.serving_scene(n, 0, seed=9)
        raw = sarsim.echo(spec)
        hr = orc.matched_filter(n, sarsim.lfm_chirp(*spec.range_chirp)).astype(np.complex64)
        ha = orc.matched_filter(n, sarsim.lfm_chirp(*spec.az_chirp)).astype(np.complex64)
        out.append(dict(n_range=n, n_az=n, pool=torch.from_numpy(raw).cuda(), range_spectrum=torch.from_numpy(hr).cuda(),
                        az_spectrum=torch.from_numpy(ha).cuda(), raw=raw, hr=hr, ha=ha, spec=spec))
    return out


def _outputs(classes, sizes):
    return [torch.full((classes[k]["n_range"], classes[k]["n_az"]), float("nan"), dtype=torch.complex64,
                       device="cuda") for k in sizes]


@pytest.mark.parametrize("size_priority,aging_s", [(False, 0.0), (True, 0.0), (True, 1e-6)],
                         ids=["one-priority", "size-priority", "size-priority-aging"])
def test_results_are_the_same_alone_and_in_the_mix(sar, classes, size_priority, aging_s):
    """With one stream priority, with smaller scenes on higher-priority
    streams (which only changes the order blocks reach the SMs), and with
    aging so short that admission is restricted most of the time (which only
    changes the admission order)."""
    rng = sarsim.uniform(21, 3, 0, 48)
    sizes = [int(u * 3) for u in rng]
    srv = sar.sar_server_create(classes, hbm_budget_bytes=1 << 30, max_inflight=8, size_priority=size_priority,
                                aging_s=aging_s)
    outs = _outputs(classes, sizes)
    res = sar.sar_server_run(srv, [(0.0, k, o) for k, o in zip(sizes, outs)], mode=sar.SAR_SERVE_CLOSED_LOOP)
    assert all(r["status"] == 0 for r in res)
    for i, k in enumerate(sizes):
        alone = _outputs(classes, [k])[0]
        r1 = sar.sar_server_run(srv, [(0.0, k, alone)], mode=sar.SAR_SERVE_CLOSED_LOOP)
        assert r1[0]["status"] == 0
        assert torch.equal(alone, outs[i]), i
    srv.destroy()


def test_server_images_match_oracle(sar, classes):
    orc = oracle.default()
    srv = sar.sar_server_create(classes, hbm_budget_bytes=1 << 30, max_inflight=4)
    outs = _outputs(classes, [0, 1, 2])
    sar.sar_server_run(srv, [(0.0, k, o) for k, o in zip([0, 1, 2], outs)], mode=sar.SAR_SERVE_CLOSED_LOOP)
    for k, o in enumerate(outs):
        c = classes[k]
        ref = orc.rda(c["raw"], c["hr"].astype(np.complex128), c["ha"].astype(np.complex128))
        img = o.cpu().numpy()
        assert M.rel_l2(img, ref) < 2e-5
        for (a0, r0) in c["spec"].targets:       # up to 16 targets: compare with the oracle's peaks
            assert M.peak(img, (r0, a0)) == M.peak(ref, (r0, a0))
    srv.destroy()


def test_budget_serialises_and_open_loop_timestamps(sar, classes):
    one = 2 * 1024 * 1024 * 8                    # footprint of one 1024^2 request
    srv = sar.sar_server_create(classes, hbm_budget_bytes=one, max_inflight=8)
    arrivals = sarsim.poisson_arrivals(3, 12, 2000.0)
    res = sar.sar_server_run(srv, [(float(t), 2) for t in arrivals], mode=sar.SAR_SERVE_OPEN_LOOP)
    assert all(r["status"] == 0 for r in res)
    for r in res:
        assert r["admit_s"] >= r["arrival_s"] - 1e-4
        assert r["done_s"] > r["admit_s"] - 1e-3
    # only one fits at a time: completions are strictly ordered and do not overlap admissions
    done = sorted(r["done_s"] for r in res)
    admits = sorted(r["admit_s"] for r in res)
    for k in range(1, len(res)):
        assert admits[k] >= done[k - 1] - 1e-3
    with pytest.raises(sar.SarError):
        sar.sar_server_create(classes, hbm_budget_bytes=one // 4)      # a class that can never fit
    srv.destroy()
