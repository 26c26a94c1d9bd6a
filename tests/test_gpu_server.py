"""Serving loop: memory-budgeted admission and continuous batching.  Every
job's result must be the same alone and in the mix (bitwise: each job owns its
tiles and partial sums), jobs larger than the budget are rejected, and jobs
that do not fit at once wait for memory and still complete."""
import threading
import time

import numpy as np
import pytest

from paper_2609_34622_b300 import synth

pytestmark = pytest.mark.gpu


def _jobs():
    rng = np.random.default_rng(81)
    jobs = []
    for i in range(4):
        x = synth.ecg_signal(int(rng.integers(3000, 9000)), 250.0, rng)
        y, sp = synth.poisson_observe(x, float(rng.uniform(5, 50)), rng)
        jobs.append((y, dict(noise=("poisson", sp), patch=(32,), step=(4,), search=(129,), group_size=(16, 32))))
    for i in range(4):
        s = int(rng.integers(40, 120))
        x = synth.disc_rect_image((s, s + 7), rng)
        y, sp = synth.poisson_observe(x, float(rng.uniform(2, 30)), rng)
        jobs.append((y, dict(noise=("poisson", sp), patch=(8, 8), step=(3, 3), search=(19, 19), group_size=(16, 32))))
    for i in range(2):
        lam = synth.ellipsoid_phantom((20, 24, 18), rng)
        y, sp = synth.poisson_observe(lam / lam.max(), 5.0, rng)
        jobs.append((y, dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2), search=(7, 7, 7),
                             group_size=(16, 32), mass_conserve=3 if i == 0 else 0)))
    x = synth.texture_edge_image((70, 90), rng)
    jobs.append((synth.gaussian_observe(x, 25 / 255, rng),
                 dict(noise=("gaussian", 25 / 255), patch=(8, 8), step=(3, 3), search=(19, 19), group_size=(16, 32))))
    return jobs


def _alone(ctx, y, cfg):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
    o = torch.empty_like(t)
    ctx.bmnd_denoise(t, o, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     cfg.get("mass_conserve", 0))
    return o.cpu().numpy()


@pytest.mark.parametrize("budget_mb,slots", [(2048, 64), (24, 3)])
def test_server_mix_equals_alone(budget_mb, slots):
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    ctx = bm.Context(0)
    jobs = _jobs()
    alone = [_alone(ctx, y, c) for y, c in jobs]
    srv = bm.Server(0, mem_budget=budget_mb << 20, max_slots=slots)
    tickets = []

    def client():
        # a burst (all jobs queued while the first steps run) with the large
        # budget; spaced arrivals with the small one
        for k, (y, c) in enumerate(jobs):
            tickets.append(srv.bmnd_server_submit(y, c))
            if slots != 64:
                time.sleep(0.002 * (k % 3))
    th = threading.Thread(target=client)
    th.start()
    th.join()
    lats = []
    for k, t in enumerate(tickets):
        out, lat = srv.bmnd_server_wait(t, 60000)
        np.testing.assert_array_equal(out, alone[k])
        lats.append(lat)
    st = srv.bmnd_server_get_stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["voxels_per_s"] > 0
    if slots == 64:
        assert st["mean_jobs_per_step"] > 1.0   # work of several jobs shared launches
    srv.close()
    ctx.close()


def test_server_rejects_oversized_and_invalid():
    import paper_2609_34622_b300.bmnd as bm
    srv = bm.Server(0, mem_budget=1 << 20, max_slots=4)
    big = np.zeros((512, 512), np.float32)
    with pytest.raises(bm.BmndError) as e:
        srv.bmnd_server_submit(big, dict(noise=("poisson", 0.1), patch=(8, 8), step=(3, 3), search=(19, 19)))
    assert e.value.status == bm.ENOMEM
    with pytest.raises(bm.BmndError) as e:
        srv.bmnd_server_submit(np.zeros(100, np.float32), dict(noise=("poisson", 0.1), patch=(8,), step=(3,),
                                                               search=(18,)))
    assert e.value.status == bm.EINVAL
    srv.close()


def test_server_large_lane_equals_alone():
    """Jobs estimated above a millisecond run in the large-job lane (one CTA
    per tile, shortest first) beside the small-job lane; each result is still
    bitwise the job alone."""
    import paper_2609_34622_b300.bmnd as bm
    rng = np.random.default_rng(83)
    jobs = _jobs()[:6]
    for i in range(2):
        x = synth.texture_edge_image((512, 512), rng)
        y, sp = synth.poisson_observe(x, 10.0, rng)
        jobs.insert(2 * i, (y, dict(noise=("poisson", sp), patch=(8, 8), step=(3, 3), search=(39, 39),
                                    group_size=(16, 32))))
    lam = synth.ellipsoid_phantom((64, 64, 64), rng)
    y, sp = synth.poisson_observe(lam / lam.max(), 3.0, rng)
    jobs.append((y, dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2), search=(11, 11, 11),
                         group_size=(16, 32), mass_conserve=3)))
    ctx = bm.Context(0)
    alone = [_alone(ctx, y, c) for y, c in jobs]
    srv = bm.Server(0, mem_budget=8 << 30, max_slots=32)
    tickets = [srv.bmnd_server_submit(y, c) for y, c in jobs]
    for k, t in enumerate(tickets):
        out, _ = srv.bmnd_server_wait(t, 120000)
        np.testing.assert_array_equal(out, alone[k])
    st = srv.bmnd_server_get_stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    srv.close()
    ctx.close()
