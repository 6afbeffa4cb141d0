"""Streaming serving: requests arriving while others run are admitted as slots
and device memory free up, run concurrently on their own streams, and every
request's result is identical to the result of running it alone and to the
CPU oracle's reconstruction of the same events (every request, the
heavy-ion-like ones included)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_05041_b300 as velo
import velogen
from _compare import assert_same, to_numpy
from paper_2412_05041_b300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    velo.build()
    assert torch.cuda.is_available()


def make_requests(n_req=24, ev_per_req=24, seed=6):
    """Pile-up-5.5 events with 5 % heavy-ion-like events (1 PV, 2000-3000 tracks)."""
    cfg = velogen.Config(seed=seed, n_events=n_req * ev_per_req, hi_frac=0.05, hi_min_tracks=2000, hi_max_tracks=3000)
    b = velogen.generate(cfg)
    reqs = []
    arrivals = serve.poisson_arrivals(n_req, rate_per_s=400.0, seed=seed)
    for i in range(n_req):
        e0, e1 = i * ev_per_req, (i + 1) * ev_per_req
        off = (b.offsets[e0:e1 + 1] - b.offsets[e0]).astype(np.uint64)
        pix = b.pixels[int(b.offsets[e0]):int(b.offsets[e1])].copy()
        reqs.append(serve.Request(i, off, pix, arrival=float(arrivals[i])))
    return reqs, b.geometry


def alone(req, geo):
    off = torch.from_numpy(req.offsets.view(np.int64)).cuda()
    pix = torch.from_numpy(req.pixels.view(np.int32)).cuda()
    return to_numpy(velo.reconstruct(off, pix, geo, velo.default_params()))


def check_same(req, geo):
    """The served result equals the request run alone (bit for bit) and the
    oracle's result on the request's events (hit lists and cluster positions
    exact, states within the 1e-5 contract)."""
    ref = alone(req, geo)
    got = to_numpy(req.result)
    for k in ("status", "cluster_offsets", "cluster_x", "cluster_y", "cluster_z", "track_offsets", "track_hit_offsets",
              "track_hits", "track_states"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"request {req.rid} {k}")
    assert_same(got, oracle.reconstruct(req.offsets, req.pixels, geo, oracle.Params()))


def test_results_identical_alone_and_in_the_mix():
    reqs, geo = make_requests()
    S = serve.Server(geo, velo.default_params(), memory_budget=40 << 30, n_slots=8)
    stats = S.run(reqs)
    assert stats["requests"] == len(reqs) and stats["max_in_flight"] > 1
    assert stats["peak_memory_bytes"] <= stats["budget_bytes"]
    n_heavy = 0
    for r in reqs:
        assert r.done >= r.admitted >= r.arrival
        check_same(r, geo)
        n_heavy += int((np.diff(r.offsets.astype(np.int64)) > 60000).sum())
    assert n_heavy > 0  # the mix holds heavy-ion-like events, and they were checked


def test_memory_budget_limits_admission():
    reqs, geo = make_requests(n_req=10, ev_per_req=16, seed=8)
    for r in reqs:
        r.arrival = 0.0  # all at once
    need = max(serve.footprint(r.n_events, len(r.pixels)) for r in reqs)
    S = serve.Server(geo, velo.default_params(), memory_budget=int(2.5 * need), n_slots=8)
    stats = S.run(reqs)
    assert stats["peak_memory_bytes"] <= stats["budget_bytes"]
    assert stats["max_in_flight"] < len(reqs)  # the budget, not the 8 slots, held requests back
    assert any(r.admitted > 0.0 for r in reqs)
    for r in reqs:
        check_same(r, geo)
    with pytest.raises(ValueError):
        serve.Server(geo, velo.default_params(), memory_budget=need // 2).run(reqs[:1])
