"""Serving loop: requests admitted while others run give the same bits as each pair alone."""
import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import scenes, serve


def test_poisson_arrivals_rate_and_order():
    t = serve.poisson_arrivals(20000, 1000.0, 3)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 1000.0) < 30.0


@pytest.mark.gpu
def test_serving_mix_equals_alone_and_oracle():
    import torch
    srv = serve.Server(n_streams=3, max_batch=4, budget_bytes=3 * 400_000_000)
    rng = np.random.default_rng(0)
    reqs = []
    t = serve.poisson_arrivals(40, 400.0, 1)
    pool = {}
    for i in range(40):
        W = int(rng.choice([64, 120, 200]))
        H = int(rng.choice([40, 80]))
        D = int(rng.choice([32, 64, 128]))
        key = (W, H, D)
        if key not in pool:
            L, R, _ = scenes.make_scene(("road", "nadir")[len(pool) % 2], len(pool), W, H, D)
            pool[key] = (L, R, torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda())
        reqs.append(serve.Request(i, float(t[i]), pool[key][2], pool[key][3], W, H, D))
    stats = srv.run(reqs)
    assert stats["requests"] == 40 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["mean_batch"] >= 1
    assert serve.check_alone(srv, reqs, range(40)) == []
    for r in reqs[::7]:
        L, R = pool[(r.W, r.H, r.D)][:2]
        ref = oracle.sgm(L, R, r.D, 9, 7, 10, 120, 8, 3)
        assert np.array_equal(r.out.cpu().numpy().view(np.uint16), ref)
    srv.close()


@pytest.mark.gpu
def test_admission_rejects_request_larger_than_stream_budget():
    import torch
    srv = serve.Server(n_streams=1, max_batch=2, budget_bytes=50_000_000)
    L = torch.zeros((400, 400), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        srv.run([serve.Request(0, 0.0, L, L, 400, 400, 256)])
    srv.close()


@pytest.mark.gpu
def test_cancelled_and_failed_requests_leave_the_rest_served():
    # host-side faults: two requests cancelled before admission, one the library refuses (D = 8
    # is not a valid disparity count); the others are served bit-exactly and the server goes on
    import torch
    srv = serve.Server(n_streams=2, max_batch=1, budget_bytes=2 * 200_000_000)
    L, R, _ = scenes.make_scene("road", 3, 120, 60, 64)
    Ld, Rd = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    reqs = [serve.Request(i, 0.001 * i, Ld, Rd, 120, 60, 64) for i in range(8)]
    reqs[2].cancel()
    reqs[5].cancel()
    reqs[4].D = 8
    stats = srv.run(reqs)
    assert [r.status for r in reqs][:4] == ["ok", "ok", "cancelled", "ok"]
    assert reqs[4].status.startswith("failed") and reqs[5].status == "cancelled"
    assert stats["served"] == 5 and stats["cancelled"] == 2 and stats["failed"] == 1
    ref = oracle.sgm(L, R, 64, 9, 7, 10, 120, 8, 3)
    for r in reqs:
        if r.status == "ok":
            assert np.array_equal(r.out.cpu().numpy().view(np.uint16), ref)
        else:
            assert r.out is None
    srv.close()


def test_request_cancel_only_while_waiting():
    r = serve.Request(0, 0.0, None, None, 8, 8, 16)
    r.status = "ok"
    r.cancel()
    assert r.status == "ok"
    r = serve.Request(1, 0.0, None, None, 8, 8, 16)
    r.cancel()
    assert r.status == "cancelled"
