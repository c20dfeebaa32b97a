"""Serving: continuous batching of (transmitter, receiver set) requests of
different sizes against a resident scene.  Each result equals the request
rendered alone; admission, cancellation, timeouts and a host-injected batch
failure behave as documented (no GPU fault is ever provoked)."""
import threading

import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, norm_err, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a GPU"
    return t


@pytest.fixture(scope="module")
def rx():
    from paper_2605_24290_gb300 import rxgs
    return rxgs


def make_server(torch, rx, K=3000, C=1, seed=501):
    rng = np.random.default_rng(seed)
    sc = S.draw_scene(rng, K)
    base = S.draw_base(rng, K, C)
    mlp = S.draw_mlp(rng, C)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W, cols_per_cta=64)
    h = upload(ctx, sc, torch, base=base, mlp_flat=S.flatten_mlp(mlp, C), C=C)
    return ctx, h, g, rng, dict(scene=sc, base=base, mlp=mlp)


def alone(ctx, rx, torch, h, tx, rxp, kind, C):
    """The request rendered on its own through per-pixel compositing."""
    n = rxp.shape[0]
    csi = torch.zeros((1, n, C, 2), device="cuda")
    rssi = torch.zeros((1, n), device="cuda") if C == 1 else None
    ctx.render(h, dev(tx[None], torch), dev(rxp, torch), n, kind | rx.OUT_CSI, csi=csi, rssi=rssi)
    ctx.sync()
    out = (rssi[0] if kind == rx.OUT_RSSI else csi[0]).cpu().numpy().reshape(-1)
    return out


@pytest.mark.parametrize("C,kind_name", [(1, "OUT_RSSI"), (2, "OUT_CSI")])
def test_each_result_equals_the_request_alone(torch, rx, oracle, C, kind_name):
    """Every served result against the oracle (MLP radiance, brute-force
    render of the request's transmitter, coherent sum), element by element
    relative to the oracle's absolute chain; and against the same request
    rendered alone on the GPU."""
    kind = getattr(rx, kind_name)
    ctx, h, g, rng, inp = make_server(torch, rx, C=C)
    ctx.serve_start(h, kind=kind, max_batch_receivers=512, max_batch_views=8, slots=2)
    reqs = []
    for i in range(36):
        n = int(np.floor(np.exp(rng.uniform(0, np.log(129)))))
        reqs.append((S.draw_points(rng, 1)[0], S.draw_points(rng, n)))
    tickets = [None] * len(reqs)

    def client(lo):
        for i in range(lo, len(reqs), 4):
            tickets[i] = ctx.serve_submit(*reqs[i])

    ths = [threading.Thread(target=client, args=(q,)) for q in range(4)]
    [t.start() for t in ths]
    [t.join() for t in ths]
    per = 1 if kind == rx.OUT_RSSI else 2 * C
    results = [ctx.serve_poll(tk, reqs[i][1].shape[0] * per, timeout_us=60_000_000)
               for i, tk in enumerate(tickets)]
    st = ctx.serve_stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] < len(reqs)            # requests were batched together
    ctx.serve_stop()
    # batches go through the visibility path (W accumulated with atomics),
    # the reference through per-pixel compositing: equal within a relative
    # 1e-4 of the request's largest output magnitude
    for (tx, rxp), got in zip(reqs, results):
        ref = alone(ctx, rx, torch, h, tx, rxp, kind, C)
        scale = np.abs(ref).max() + 1e-30
        assert float(np.abs(got - ref).max()) <= 1e-4 * scale
    # the oracle: radiance of the request's receivers, the transmitter's view
    # rendered brute force, CSI / RSSI as coherent sums over the grid
    sc = inp["scene"]
    for i, ((tx, rxp), got) in enumerate(zip(reqs, results)):
        rad = oracle.mlp_radiance(inp["mlp"], rxp, sc.means, inp["base"])
        o = oracle.render_view(g, sc, tx, rad)
        a_csi = o["absacc"].sum(axis=(1, 2))                     # [n, C]
        if kind == rx.OUT_RSSI:
            e = float((np.abs(got - oracle.rssi(o["spectra"])) / (a_csi[:, 0] + 1e-30)).max())
        else:
            e = norm_err(got.reshape(-1, C, 2), oracle.csi(o["spectra"]), a_csi)
        assert e <= TOL, f"request {i} ({rxp.shape[0]} receivers): normalised error {e}"


def test_admission_cancel_timeout_and_fault(torch, rx):
    ctx, h, g, rng, _ = make_server(torch, rx, seed=502)
    ctx.serve_start(h, kind=rx.OUT_RSSI, max_batch_receivers=256, max_batch_views=4,
                    mem_budget=64 << 20, slots=1)
    # larger than a batch, and larger than the memory budget
    with pytest.raises(rx.RxgsError) as ei:
        ctx.serve_submit(S.draw_points(rng, 1)[0], S.draw_points(rng, 300))
    assert ei.value.status == rx.E_ADMISSION
    with pytest.raises(rx.RxgsError) as ei:
        ctx.serve_submit(S.draw_points(rng, 1)[0], S.draw_points(rng, 250 * 100)[:250])
        ctx.serve_submit(S.draw_points(rng, 1)[0], np.zeros((0, 3), np.float32))
    assert ei.value.status in (rx.E_ADMISSION, rx.E_INVALID)
    with pytest.raises(rx.RxgsError) as ei:
        ctx.serve_poll(123456789, 1, timeout_us=0)
    assert ei.value.status == rx.E_INVALID
    # a host-injected failure fails one batch; later requests are served
    ctx.serve_inject_fault(1)
    t_bad = ctx.serve_submit(S.draw_points(rng, 1)[0], S.draw_points(rng, 5))
    with pytest.raises(rx.RxgsError) as ei:
        ctx.serve_poll(t_bad, 5, timeout_us=30_000_000)
    assert ei.value.status == rx.E_DEVICE
    # many queued requests: cancel the last; poll with no wait
    tks = [ctx.serve_submit(S.draw_points(rng, 1)[0], S.draw_points(rng, 64)) for _ in range(30)]
    try:
        ctx.serve_cancel(tks[-1])
        cancelled = True
    except rx.RxgsError as e:
        assert e.status == rx.E_NOT_READY
        cancelled = False
    try:
        ctx.serve_poll(tks[0], 64, timeout_us=0)
    except rx.RxgsError as e:
        assert e.status == rx.E_NOT_READY
        ctx.serve_poll(tks[0], 64, timeout_us=30_000_000)
    for tk in tks[1:-1]:
        ctx.serve_poll(tk, 64, timeout_us=30_000_000)
    if cancelled:
        with pytest.raises(rx.RxgsError) as ei:
            ctx.serve_poll(tks[-1], 64, timeout_us=0)
        assert ei.value.status == rx.E_CANCELLED
    else:
        ctx.serve_poll(tks[-1], 64, timeout_us=30_000_000)
    st = ctx.serve_stats()
    assert st["failed"] == 1 and st["p99_ms"] >= st["p50_ms"] > 0
    ctx.serve_stop()
