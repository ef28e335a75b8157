"""Continuous-batching request server: results alone vs. in the mix (images
from 64^2 to 2048^2), iteration-level batching of same-size solves on and
off, budget admission, cancellation, input checks, and the device-memory
estimate."""
import math

import numpy as np
import pytest
import torch

from paper_1406_0359_gb300 import synth
from tests._gpu import need_gpu, rel

pytestmark = pytest.mark.gpu

MIX = [(64, 3000, 11), (128, 20000, 12), (256, 60000, 13), (64, 5000, 14), (128, 9000, 15), (256, 130000, 16),
       (2048, 65536, 17)]


def problem(n, M, seed):
    from paper_1406_0359_gb300.binding import Operator

    uv = synth.uv_coverage(M, n, seed)
    x = synth.sky(n, seed, 3, 10)
    op = Operator(torch.as_tensor(uv).cuda(), n, 3, "fp32")
    y0 = op.phi(torch.as_tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.complex128)
    op.close()
    a, b = synth.noise_draws(M, seed)
    sigma = np.linalg.norm(y0) / math.sqrt(M) * 10 ** (-1.5)
    y = y0 + sigma / math.sqrt(2) * (a + 1j * b)
    eps = sigma * math.sqrt(M + 2 * math.sqrt(M))
    return uv, y, eps


def run_server(reqs, slots, budget=int(40e9), batching=True, counts=None, **kw):
    from paper_1406_0359_gb300.binding import Server

    srv = Server(budget, slots)
    srv.set_batching(batching)
    kw = dict(dict(t_max=15, cg_iters=8, n_reweight=1), **kw)
    ids = [srv.submit(uv, y, n, 3, eps, **kw) for (n, uv, y, eps) in reqs]
    max_active = 0
    for _ in range(100000):
        a, q = srv.step()
        max_active = max(max_active, a)
        if a == 0 and q == 0:
            break
    out = [srv.result(i) for i in ids]
    if counts is not None:
        counts.extend(srv.counts())
    srv.close()
    return out, max_active


def test_results_same_alone_and_in_mix():
    need_gpu()
    reqs = []
    for n, M, seed in MIX:
        uv, y, eps = problem(n, M, seed)
        reqs.append((n, uv, y, eps))
    alone = [run_server([r], 1)[0][0] for r in reqs]
    mixed, max_active = run_server(reqs, 8)
    assert max_active >= 4
    for a, m in zip(alone, mixed):
        assert a is not None and m is not None
        assert m[1]["iterations"] == a[1]["iterations"] == 30
        assert rel(m[0], a[0]) < 1e-5
        assert m[2] >= m[3] >= 0.0


@pytest.mark.parametrize("xi", [0.0, 1e-3])
def test_batched_groups_equal_solo_iterations(xi):
    """Same-size solves advance in batched groups (one launch per pass over
    the group); each result equals the same server's result with batching
    off, with a fixed iteration count and with the halting test (solves of
    one group stop at different iterations and the group re-forms)."""
    need_gpu()
    reqs = [(n, *problem(n, M, seed)) for n, M, seed in
            [(128, 20000, 51), (128, 9000, 52), (64, 3000, 53), (128, 40000, 54), (64, 6000, 55), (256, 60000, 56)]]
    kw = dict(t_max=40, xi=xi) if xi else {}
    cb, cs = [], []
    on, _ = run_server(reqs, 8, batching=True, counts=cb, **kw)
    off, _ = run_server(reqs, 8, batching=False, counts=cs, **kw)
    assert cb[0] > 0 and cs[0] == 0  # groups formed only with batching on
    assert cb[0] + cb[1] == cs[1]  # the same solve-iterations in total
    for a, b in zip(on, off):
        assert a is not None and b is not None
        assert a[1]["iterations"] == b[1]["iterations"]
        if not xi:
            assert a[1]["iterations"] == 30
        assert rel(a[0], b[0]) < 1e-5


def test_cancel_member_of_a_batched_group():
    need_gpu()
    from paper_1406_0359_gb300.binding import PurifyError, Server

    reqs = [(128, *problem(128, M, s)) for M, s in ((20000, 61), (9000, 62), (30000, 63))]
    alone, _ = run_server([reqs[2]], 1, t_max=40, n_reweight=0)
    srv = Server(int(40e9), 4)
    srv.set_batching(True)
    ids = [srv.submit(uv, y, n, 3, eps, t_max=40, cg_iters=8, n_reweight=0) for (n, uv, y, eps) in reqs]
    for _ in range(6):  # all three admitted, a few batched iterations in
        srv.step()
    assert srv.counts()[0] > 0
    srv.cancel(ids[0])  # its iteration may be in flight in the group
    for _ in range(100000):
        a, q = srv.step()
        if a == 0 and q == 0:
            break
    with pytest.raises(PurifyError) as e:
        srv.result(ids[0])
    assert e.value.code == -7
    for rid in ids[1:]:
        x, st, _, _ = srv.result(rid)
        assert st["iterations"] == 40 and np.all(np.isfinite(x))
    x, st, _, _ = srv.result(ids[2])
    assert rel(x, alone[0][0]) < 1e-5
    srv.close()


def test_budget_limits_admission():
    need_gpu()
    from paper_1406_0359_gb300.binding import PurifyError, Server, purify_estimate_bytes

    reqs = [(128, *problem(128, 20000, s)) for s in (21, 22, 23)]
    one = purify_estimate_bytes(20000, 128, 3)
    _, max_active = run_server(reqs, 8, budget=int(one * 1.5))
    assert max_active == 1
    _, max_active = run_server(reqs, 8, budget=int(one * 3.5))
    assert max_active == 3
    srv = Server(int(one * 0.1), 4)
    with pytest.raises(PurifyError):
        srv.submit(reqs[2][1], reqs[2][2], reqs[2][0], 3, reqs[2][3])
    srv.close()


def test_estimate_bounds_operator_memory():
    need_gpu()
    from paper_1406_0359_gb300.binding import Operator, purify_estimate_bytes

    for n, M, seed in MIX[:3]:
        uv, y, eps = problem(n, M, seed)
        op = Operator(torch.as_tensor(uv).cuda(), n, 3, "fp32")
        op.solve(torch.as_tensor(y, dtype=torch.complex64).cuda(), eps, t_max=2, cg_iters=2)
        assert op.info()["device_bytes"] <= purify_estimate_bytes(M, n, 3)
        op.close()


def test_cancel_queued_and_running_requests():
    need_gpu()
    from paper_1406_0359_gb300.binding import PurifyError, Server

    reqs = [(128, *problem(128, 20000, s)) for s in (31, 32, 33)]
    srv = Server(int(40e9), 1)
    ids = [srv.submit(uv, y, n, 3, eps, t_max=200, cg_iters=8) for (n, uv, y, eps) in reqs]
    for _ in range(5):  # request 0 admitted and a few iterations in
        srv.step()
    srv.cancel(ids[1])  # still queued
    srv.cancel(ids[0])  # running: stopped between iterations
    with pytest.raises(PurifyError):
        srv.cancel(ids[0])  # already finished
    for _ in range(100000):
        a, q = srv.step()
        if a == 0 and q == 0:
            break
    for rid in ids[:2]:
        with pytest.raises(PurifyError) as e:
            srv.result(rid)
        assert e.value.code == -7
    x, st, lat, qs = srv.result(ids[2])  # the one left runs to the end
    assert st["iterations"] == 200 and np.all(np.isfinite(x))
    srv.close()


def test_nonfinite_request_is_refused_at_submit():
    need_gpu()
    from paper_1406_0359_gb300.binding import PurifyError, Server

    n, (uv, y, eps) = 64, problem(64, 3000, 41)
    srv = Server(int(40e9), 2)
    y = np.array(y, copy=True)
    y[123] = np.nan
    with pytest.raises(PurifyError) as e:
        srv.submit(uv, y, n, 3, eps)
    assert e.value.code == -1 and "visibility 123" in str(e.value)
    uv = np.array(uv, copy=True)
    uv[7, 0] = np.inf
    with pytest.raises(PurifyError):
        srv.submit(uv, np.zeros(3000, np.complex64), n, 3, eps)
    srv.close()
