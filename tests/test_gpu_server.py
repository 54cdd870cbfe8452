"""Continuous-batching server: results are bitwise the same alone and in a mix
of concurrent requests of other sizes, lengths and methods; the memory budget
holds (spectra evicted when needed); validation and latency reporting."""
import numpy as np
import pytest

import fsp_inputs as I
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _req(N, seed, dtype="f32"):
    import torch
    rho = to_dev(I.gaussian_mixture(N, seed=seed).astype(np.float32), dtype)
    return rho, torch.full_like(rho, float("nan"))


def test_same_result_alone_and_in_the_mix(fsp):
    import torch
    srv = fsp.Server(budget_bytes=8 << 30, max_slots=6)
    rho, alone = _req(64, 1)
    srv.wait(srv.submit(rho, alone, L=2.0, algo="vg_dct"))
    # the same request again, amid concurrent requests of other sizes/methods
    mix = []
    rng = np.random.default_rng(2407)
    for i in range(24):
        N = int(rng.choice([32, 64, 96, 128]))
        r, f = _req(N, 100 + i)
        mix.append((srv.submit(r, f, L=float(rng.choice([1.0, 2.0])), algo=str(rng.choice(["he", "vg_dct"]))), r, f))
    again = torch.full_like(alone, float("nan"))
    t = srv.submit(rho, again, L=2.0, algo="vg_dct")
    for tk, _, _ in mix:
        srv.wait(tk)
    lat = srv.wait(t)
    assert lat > 0
    assert torch.equal(alone, again)
    # and equal to a plain plan solve of the same request
    p = fsp.Plan(64, 2.0, "vg_dct", "f32")
    assert torch.equal(p.solve(rho), alone)
    st = srv.stats()
    assert st["completed"] == 26 and st["queued"] == 0 and st["running"] == 0
    assert st["spec_hits"] >= 1
    srv.close()


def test_budget_is_respected_with_eviction(fsp):
    # room for one N=64 FP32 workspace (3*64*64*80 complex) and one N=64
    # spectrum (65*65*80 reals + roots): a second spectrum forces an eviction
    ws64 = 3 * 64 * 64 * 80 * 8
    spec64 = 65 * 65 * 80 * 4 + 3 * 64 * 8
    budget = ws64 + spec64 + 400_000
    srv = fsp.Server(budget_bytes=budget, max_slots=2)
    reqs = []
    for i, (N, L) in enumerate([(64, 1.0), (64, 2.0), (32, 1.0), (64, 1.0), (64, 2.0), (32, 2.0)]):
        r, f = _req(N, i)
        reqs.append((srv.submit(r, f, L=L, algo="he"), N, L, r, f))
    for tk, *_ in reqs:
        srv.wait(tk)
        st = srv.stats()
        assert st["bytes_in_use"] <= budget
    assert srv.stats()["evictions"] >= 1
    for tk, N, L, r, f in reqs:
        ref = fsp.Plan(N, L, "he", "f32").solve(r)
        assert bool((ref == f).all())
    srv.close()


def test_server_validation(fsp):
    srv = fsp.Server(budget_bytes=1 << 30, max_slots=1)
    r, f = _req(14, 0)  # 2N = 28 is not 2/3/5-smooth
    with pytest.raises(fsp.FspError):
        srv.submit(r, f)
    with pytest.raises(fsp.FspError):
        srv.poll(123456)
    srv.close()
    with pytest.raises(fsp.FspError):
        fsp.Server(budget_bytes=0)


def test_request_larger_than_budget_fails_cleanly(fsp):
    srv = fsp.Server(budget_bytes=1 << 20, max_slots=1)  # 1 MB: no N=64 workspace fits
    r, f = _req(64, 0)
    t = srv.submit(r, f)
    with pytest.raises(fsp.FspError):
        srv.wait(t)
    r2, f2 = _req(8, 0)  # small requests still go through
    assert srv.wait(srv.submit(r2, f2)) > 0
    srv.close()


def test_small_request_completes_while_a_spectrum_is_built(fsp):
    """A cold N = 256 Vico-Greengard (DCT route) request starts a spectrum build
    of about 100 ms on the builder thread; a warm N = 32 request submitted just
    after it is admitted and finished meanwhile, within a few ms, and the
    budget (spectra + workspaces + the build's reserved temporaries) holds."""
    import torch
    budget = 6 << 30
    srv = fsp.Server(budget_bytes=budget, max_slots=4)
    small, fs = _req(32, 5)
    srv.wait(srv.submit(small, fs, L=1.0, algo="he"))  # its spectrum is now cached
    big, fb = _req(256, 6)
    t_big = srv.submit(big, fb, L=1.0, algo="vg_dct")
    t_small = srv.submit(small, torch.full_like(fs, float("nan")), L=1.0, algo="he")
    lat_small = srv.wait(t_small)
    st = srv.stats()
    big_state = srv.poll(t_big)[0]
    lat_big = srv.wait(t_big)
    print("N=32 latency %.2f ms while the N=256 build ran (big state then %d), N=256 latency %.1f ms, "
          "peak bytes %.3f GB" % (lat_small, big_state, lat_big, st["peak_bytes_in_use"] / 1e9))
    assert big_state < srv.DONE and st["builds_in_flight"] >= 1  # the build was still going
    assert lat_small < 20.0
    assert lat_big > lat_small
    assert srv.stats()["peak_bytes_in_use"] <= budget
    ref = fsp.Plan(256, 1.0, "vg_dct", "f32").solve(big)
    assert torch.equal(ref, fb)
    srv.close()


def test_vg_build_larger_than_budget_is_refused(fsp):
    """FSP_VG builds its kernel on the (4N)^3 grid: at N = 128 that is 2.1 GB
    of temporaries, refused under a 1 GB budget; the DCT route fits."""
    srv = fsp.Server(budget_bytes=1 << 30, max_slots=2)
    r, f = _req(128, 1)
    with pytest.raises(fsp.FspError) as ei:
        srv.wait(srv.submit(r, f, algo="vg"))
    assert ei.value.status == fsp.FSP_ENOMEM
    assert srv.wait(srv.submit(r, f, algo="vg_dct")) > 0
    assert srv.stats()["peak_bytes_in_use"] <= 1 << 30
    srv.close()
