"""Benchmark: receiver spectra per second, batched vs a per-receiver loop.

Workload (one step = the whole hot path over one batch):
  100,000 Gaussians in a 10x8x3 m box, 32 transmitters x 64 receivers,
  radiance from the 2-layer 64-wide conditioning MLP, 90x360 grid, 16x16
  tiles.  A step = transmitter-side preparation (projection, key emission,
  radix sort, tile ranges), MLP radiance, compositing into 2,048 spectra plus
  their CSI/RSSI reduction, and the backward pass to opacity, phi_base and
  the MLP weights for an N(0,1) cotangent on the spectra.
  value = spectra per second = 2,048 / step time (inputs resident in HBM).

Also reported: the per-receiver loop (the same kernels, one (tx, rx) pair per
call, the full pipeline per pair), the end-to-end figure through the C ABI
with host buffers (pinned H2D of the step's inputs, D2H of its gradients and
RSSI), the roofline of the dominant kernel, clocks during the timed region
and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own GPU (independent
transmitter batches; no collective on the data path) and rank 0 prints the
whole-job throughput.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "receiver spectra/sec batched vs per-rx loop, same GB300; p50/p99 serve ms"
UNIT = "spectra/s"
WORKLOAD = "100k Gaussians, 32 tx x 64 rx, MLP radiance (2-layer, 64 wide), 90x360 grid, fwd+bwd"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch,
# measured by one ncu capture of that kernel on this workload; valid only
# while the kernel sources hash to the value recorded at capture time.
NCU_TRAFFIC = {
    "render_fwd": {"bytes": 19_888_896 + 483_264_000, "tile": [8, 32], "cols": 128,
                   "files": ['render_fwd_tc.cu', 'render_common.cuh', 'rxgs_math.cuh', 'tc_common.cuh'],
                   "sha1": "822d37bb986e6847"},
    "render_bwd": {"bytes": 561_249_024 + 8_143_360, "tile": [8, 32], "cols": 128,
                   "files": ['render_bwd_tc.cu', 'render_common.cuh', 'rxgs_math.cuh', 'tc_common.cuh'],
                   "sha1": "5fc5890331f1f8c7"},
}


def ncu_traffic(kernel, tile, cols):
    import hashlib
    e = NCU_TRAFFIC.get(kernel)
    if not e or list(tile) != e["tile"] or cols != e["cols"]:
        return None
    m = hashlib.sha1()
    for f in e["files"]:
        with open(os.path.join(ROOT, "paper_2605_24290_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return e["bytes"] if m.hexdigest()[:16] == e["sha1"] else None


def fp32_alu_peak_tflops(sm_mhz, sms):
    """SMs x 128 FP32 lanes x 2 flops per FMA x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.idx = gpu_index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def whole_job_rate(torch, dist, ms_local, units_per_step, device):
    """Replicas: every rank processes `units_per_step` per step in
    `ms_local` ms; the job's step time is the slowest rank's (max over
    ranks) and its rate counts the units of all ranks.  Returns
    (ms_max, units per second of the whole job)."""
    t = torch.tensor([float(ms_local)], device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return ms_max, world * units_per_step / (ms_max / 1e3)


# --------------------------------------------------------------- the step
class Workload:
    def __init__(self, torch, rxgs, S, device, tile=None, cols=0):
        self.torch = torch
        w = S.workload_mlp()
        self.w = w
        g, sc, C = w["grid"], w["scene"], w["C"]
        self.g, self.C = g, C
        self.M, self.N, self.K = w["tx"].shape[0], w["rx"].shape[0], sc.K
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        th, tw = tile if tile else (16, 16)
        self.ctx = rxgs.Context(H=g.H, W=g.W, tile_h=th, tile_w=tw, cols_per_cta=cols)
        self.rxgs = rxgs
        flat = S.flatten_mlp(w["mlp"], C)
        self.nmlp = flat.shape[0]
        self.scene = self.ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats),
                                           d(sc.opacity), d(w["base"]), d(flat), C=C)
        self.tx, self.rx = d(w["tx"]), d(w["rx"])
        M, N, K = self.M, self.N, self.K
        self.spec = torch.empty((M, N, g.H, g.W, C, 2), device=device)
        self.csi = torch.empty((M, N, C, 2), device=device)
        self.rssi = torch.empty((M, N), device=device)
        gen = torch.Generator(device=device)
        gen.manual_seed(S.SEED_BASE + 1)
        self.gspec = torch.randn((M, N, g.H, g.W, C, 2), device=device, generator=gen)
        self.d_tau = torch.zeros(K, device=device)
        self.d_base = torch.zeros((K, C, 2), device=device)
        self.d_mlp = torch.zeros(self.nmlp, device=device)
        self.kind = rxgs.OUT_SPECTRA | rxgs.OUT_CSI | rxgs.OUT_RSSI

    def step(self, tx=None, rx=None, gspec=None, before_backward=None, spec=None, rssi=None):
        c, rx_ = self.ctx, self.rxgs
        tx = self.tx if tx is None else tx
        rx = self.rx if rx is None else rx
        gspec = self.gspec if gspec is None else gspec
        spec = self.spec if spec is None else spec
        rssi = self.rssi if rssi is None else rssi
        views = c.prepare(self.scene, tx)
        c.render_views(views, rx, self.N, self.kind, spectra=spec, csi=self.csi, rssi=rssi)
        if before_backward is not None:
            before_backward()
        self.d_tau.zero_()
        self.d_base.zero_()
        self.d_mlp.zero_()
        c.render_backward(views, rx, self.N, rx_.OUT_SPECTRA, grad_spectra=gspec,
                          grad_opacity=self.d_tau, grad_base=self.d_base, grad_mlp=self.d_mlp)
        c.release_views(views)

    def loop_pair(self, i, j, spec1, g1):
        """One (tx, rx) pair through the full pipeline, forward + backward."""
        c, rx_ = self.ctx, self.rxgs
        views = c.prepare(self.scene, self.tx[i:i + 1])
        c.render_views(views, self.rx[j:j + 1], 1, rx_.OUT_SPECTRA, spectra=spec1)
        c.render_backward(views, self.rx[j:j + 1], 1, rx_.OUT_SPECTRA, grad_spectra=g1,
                          grad_opacity=self.d_tau, grad_base=self.d_base, grad_mlp=self.d_mlp)
        c.release_views(views)

    def composited_pairs(self):
        """Number of (pixel, Gaussian) pairs composited per step (each
        transmitter's pixels x the Gaussians each pixel composites)."""
        t = self.torch
        ncon = t.zeros((self.M, self.g.H, self.g.W), dtype=t.int32, device=self.tx.device)
        views = self.ctx.prepare(self.scene, self.tx)
        self.ctx.render_views(views, self.rx, self.N, self.rxgs.OUT_SPECTRA, spectra=self.spec,
                              ncontrib=ncon)
        self.ctx.release_views(views)
        return int(ncon.sum().item())


def bench_config(world):
    """The workload of one step, shared by both arms of the benchmark."""
    return {"workload": WORKLOAD, "gaussians": 100_000, "transmitters": 32, "receivers": 64,
            "grid": [90, 360], "spectra_per_step": 32 * 64,
            "step": "prepare + MLP + forward (spectra, CSI, RSSI) + backward",
            "l2": "flushed between timed steps (256 MB write)",
            "parallelism": f"replicas x{world}"}


def l2_flush(torch, buf):
    buf.add_(1.0)


def gpu_bench(args):
    import torch
    import torch.distributed as dist

    from paper_2605_24290_gb300 import rxgs
    from paper_2605_24290_gb300 import synthetic as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = Workload(torch, rxgs, S, dev, tile=args.tile, cols=args.cols)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    tune = None
    if not args.no_tune and not args.tile:
        # the project's autotuner picks tile shape and columns per CTA on
        # this workload (forward pass); the choice stays in the context
        tune = W.ctx.autotune(W.scene, W.tx, W.rx, W.N, W.kind, iters=2)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        W.step()
    barrier()
    # ---- timed region: K steps, per-step CUDA events, L2 flushed between steps
    stream = torch.cuda.current_stream()
    W.ctx.profile(True)
    W.ctx.profile_read(reset=True)
    launches0 = W.ctx.profile_read(reset=False)["kernel_launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            l2_flush(torch, flush)
            evs[k][0].record(stream)
            W.step()
            evs[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
    prof = W.ctx.profile_read(reset=True)
    W.ctx.profile(False)
    launches = prof["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    spectra_per_step = W.M * W.N
    ms_max, value = whole_job_rate(torch, dist if world > 1 else None, ms, spectra_per_step, dev)

    # ---- roofline of the dominant kernel
    stages = prof["stages"]
    calls = max(1, stages.get("render_fwd", {}).get("calls", 1))
    dom = max(stages.items(), key=lambda kv: kv[1]["ms"])[0] if stages else "render_fwd"
    P = W.composited_pairs()
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_alu_peak_tflops(sm_mhz, sms)
    tile = tune["chosen"]["tile"] if tune else (list(args.tile) if args.tile else [16, 16])
    # column block of the forward (the backward always takes 128 for 128 columns)
    cols = tune["chosen"]["cols"] if tune else (
        args.cols if args.cols else (128 if 2 * W.N * W.C > 64 else 64))

    def roofline(kernel, flops_per_pair, what):
        if kernel not in stages:
            return None
        kms = stages[kernel]["ms"] / stages[kernel]["calls"]
        ach = P * flops_per_pair / (kms / 1e3) / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": ncu_traffic(kernel, tile, cols if kernel == "render_fwd" else 128),
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({src} clock)",
                "units": f"{P} composited (pixel, Gaussian) pairs x {what} flops",
                "launch_ms": round(kms, 4)}

    # dominant kernel: the backward (weight 16 + gamma 4NC + dL/ds 4NC per pair)
    roof = roofline("render_bwd", 16 + 8 * W.N * W.C, "(16 + 8*N*C)")
    roof_fwd = roofline("render_fwd", 16 + 4 * W.N * W.C, "(16 + 4*N*C)")

    # ---- per-receiver loop on a bounded sample of pairs (same kernels)
    loop = None
    if rank == 0 and not args.no_loop:
        spec1 = torch.empty((1, 1, W.g.H, W.g.W, W.C, 2), device=dev)
        g1 = W.gspec[0:1, 0:1].contiguous()
        pairs = [(i % W.M, (7 * i) % W.N) for i in range(args.loop_pairs)]
        for (i, j) in pairs[:3]:
            W.loop_pair(i, j, spec1, g1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for (i, j) in pairs:
            W.loop_pair(i, j, spec1, g1)
        b.record()
        torch.cuda.synchronize()
        lms = a.elapsed_time(b)
        loop = {"value": round(len(pairs) / (lms / 1e3), 2), "unit": UNIT,
                "sample": f"{len(pairs)} (tx, rx) pairs, each prepare + MLP + forward + backward",
                "ms_per_pair": round(lms / len(pairs), 4),
                "batched_over_loop": round((spectra_per_step / (ms_max / 1e3)) / (len(pairs) / (lms / 1e3)), 2)}
        # stricter loop: each transmitter's view prepared (projected, sorted)
        # once outside the timed region; per pair only MLP + forward + backward
        c, rx_ = W.ctx, W.rxgs
        vmap = {i: c.prepare(W.scene, W.tx[i:i + 1]) for i in sorted({i for i, _ in pairs})}

        def render_pair(i, j):
            c.render_views(vmap[i], W.rx[j:j + 1], 1, rx_.OUT_SPECTRA, spectra=spec1)
            c.render_backward(vmap[i], W.rx[j:j + 1], 1, rx_.OUT_SPECTRA, grad_spectra=g1,
                              grad_opacity=W.d_tau, grad_base=W.d_base, grad_mlp=W.d_mlp)

        for (i, j) in pairs[:3]:
            render_pair(i, j)
        torch.cuda.synchronize()
        a.record()
        for (i, j) in pairs:
            render_pair(i, j)
        b.record()
        torch.cuda.synchronize()
        rms = a.elapsed_time(b)
        for vh in vmap.values():
            c.release_views(vh)
        loop["render_only"] = {
            "value": round(len(pairs) / (rms / 1e3), 2), "unit": UNIT,
            "sample": f"{len(pairs)} pairs; views prepared once per transmitter outside the timing",
            "ms_per_pair": round(rms / len(pairs), 4),
            "batched_over_loop": round((spectra_per_step / (ms_max / 1e3)) / (len(pairs) / (rms / 1e3)), 2)}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_tx = torch.from_numpy(W.w["tx"]).pin_memory()
        h_rx = torch.from_numpy(W.w["rx"]).pin_memory()
        h_g = torch.empty(W.gspec.shape, dtype=torch.float32).pin_memory()
        h_g.copy_(W.gspec.cpu())
        d_tx, d_rx = torch.empty_like(W.tx), torch.empty_like(W.rx)
        d_g = torch.empty_like(W.gspec)
        o_tau = torch.empty(W.K).pin_memory()
        o_base = torch.empty((W.K, W.C, 2)).pin_memory()
        o_mlp = torch.empty(W.nmlp).pin_memory()
        o_rssi = torch.empty((W.M, W.N)).pin_memory()
        o_spec = torch.empty(W.spec.shape).pin_memory()
        h2d = h_tx.numel() * 4 + h_rx.numel() * 4 + h_g.numel() * 4
        d2h = (o_tau.numel() + o_base.numel() + o_mlp.numel() + o_rssi.numel() +
               o_spec.numel()) * 4

        # Every step copies its own inputs in and its results out, through
        # two copy streams (copies in one direction share a copy engine in
        # issue order, so nothing small is queued behind a large copy): step
        # k + 1's tx, rx and then its cotangent (531 MB, needed only by the
        # backward) go up while step k computes, into the other of two device
        # buffers; step k's spectra come down while its backward and the
        # next forward run (with its RSSI), and its gradients after its
        # backward.
        copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
        d_txs = [d_tx, torch.empty_like(W.tx)]
        d_rxs = [d_rx, torch.empty_like(W.rx)]
        d_gs = [d_g, torch.empty_like(W.gspec)]
        specs = [W.spec, torch.empty_like(W.spec)]
        rssis = [W.rssi, torch.empty_like(W.rssi)]
        ev = lambda: [torch.cuda.Event(), torch.cuda.Event()]
        ev_in, ev_g, ev_bwd, ev_out, ev_small = ev(), ev(), ev(), ev(), ev()

        def upload(k):
            b = k % 2
            if k >= 2:
                copy_in.wait_event(ev_bwd[b])  # step k - 2 is done with buffers b
            with torch.cuda.stream(copy_in):
                d_txs[b].copy_(h_tx, non_blocking=True)
                d_rxs[b].copy_(h_rx, non_blocking=True)
                ev_in[b].record(copy_in)
                d_gs[b].copy_(h_g, non_blocking=True)
                ev_g[b].record(copy_in)

        def e2e_step(k, last):
            cur = torch.cuda.current_stream()
            b = k % 2
            if k >= 2:
                cur.wait_event(ev_out[b])  # the spectra of step k - 2 are down
            cur.wait_event(ev_in[b])
            if not last:
                upload(k + 1)

            def before_backward():
                f_done = torch.cuda.Event()
                f_done.record(cur)
                copy_out.wait_event(f_done)
                with torch.cuda.stream(copy_out):
                    o_spec.copy_(specs[b], non_blocking=True)
                    o_rssi.copy_(rssis[b], non_blocking=True)
                    ev_out[b].record(copy_out)
                cur.wait_event(ev_g[b])
                if k >= 1:
                    cur.wait_event(ev_small[1 - b])  # step k - 1's gradients are down

            W.step(d_txs[b], d_rxs[b], d_gs[b], before_backward=before_backward, spec=specs[b],
                   rssi=rssis[b])
            ev_bwd[b].record(cur)
            copy_out.wait_event(ev_bwd[b])
            with torch.cuda.stream(copy_out):
                o_tau.copy_(W.d_tau, non_blocking=True)
                o_base.copy_(W.d_base, non_blocking=True)
                o_mlp.copy_(W.d_mlp, non_blocking=True)
                ev_small[b].record(copy_out)

        def e2e_run(n):
            upload(0)
            for k in range(n):
                e2e_step(k, k == n - 1)
            torch.cuda.synchronize()

        e2e_run(2)
        n_e = max(20, args.steps)
        barrier()
        t0 = time.perf_counter()
        e2e_run(n_e)
        barrier()
        e_ms = (time.perf_counter() - t0) * 1e3 / n_e
        e_ms, e_val = whole_job_rate(torch, dist if world > 1 else None, e_ms, spectra_per_step,
                                     dev)
        # this machine's host links with the same pinned buffers and streams:
        # the cotangent up alone, the spectra down alone, both at once (best
        # of three each); (up + down bytes) / both-at-once is the copy bound
        # of one e2e step
        def link_ms(up, down):
            best = float("inf")
            for _ in range(3):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                if up:
                    with torch.cuda.stream(copy_in):
                        d_gs[1].copy_(h_g, non_blocking=True)
                if down:
                    with torch.cuda.stream(copy_out):
                        o_spec.copy_(specs[1], non_blocking=True)
                torch.cuda.synchronize()
                best = min(best, (time.perf_counter() - t1) * 1e3)
            return best

        up_b, down_b = h_g.numel() * 4, o_spec.numel() * 4
        t_up, t_down, t_both = link_ms(True, False), link_ms(False, True), link_ms(True, True)
        link = {"h2d_gbs": round(up_b / t_up / 1e6, 1), "d2h_gbs": round(down_b / t_down / 1e6, 1),
                "both_gbs": round((up_b + down_b) / t_both / 1e6, 1),
                "copy_bound_ms": round((h2d + d2h) / ((up_b + down_b) / t_both) , 4)}
        e2e = {"value": round(e_val, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(e_ms, 4), "host_links": link,
               "copies": "H2D tx, rx and the spectra cotangent; D2H the spectra, RSSI and the "
                         "opacity, phi_base and MLP gradients (pinned host buffers); the next "
                         "step's cotangent goes up and this step's spectra come down on two copy "
                         "streams while the GPU computes"}

    serve = None
    if rank == 0 and not args.no_serve:
        serve = serve_bench(torch, rxgs, S, seconds=args.serve_seconds)
    bcsi = None
    if rank == 0 and not args.no_batched:
        bcsi = batched_csi_bench(torch, rxgs, S)
    cov = None
    if rank == 0 and not args.no_coverage:
        cov = coverage_bench(torch, rxgs, S, K=args.coverage_gaussians)
    fle = None
    if rank == 0 and not args.no_fle:
        fle = fle_bench(torch, rxgs, S, K=args.fle_gaussians)
    train = None
    if rank == 0 and not args.no_train:
        train = train_bench(torch, rxgs, S)
    occ = None
    if rank == 0 and not args.no_occupancy:
        occ = occupancy_bench(torch, rxgs, S, W)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_sample(args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; indoor-room scene recipe)",
            "config": dict(bench_config(world), tile_autotuned=tune["chosen"] if tune else None,
                           tile=tile, cols=cols),
            "wall_s": round(wall, 3),
            "stages_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in stages.items()},
            "dominant_stage": dom,
            "autotune": tune,
            "roofline": roof,
            "roofline_fwd": roof_fwd,
            "per_rx_loop": loop,
            "serve": serve,
            "batched_csi": bcsi,
            "coverage": cov,
            "fle": fle,
            "train_step": train,
            "occupancy": occ,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- serving
def serve_bench(torch, rxgs, S, seconds=60.0, rate=200.0, warm=3.0, sweep_factors=(0.5, 2.0, 4.0),
                sweep_seconds=3.0):
    """300,000 resident Gaussians (MLP radiance), Poisson requests at `rate`
    per second, each 1 transmitter and n = floor(exp(U(0, ln 1025))) receivers,
    RSSI out; latency = submit to completion (library-side)."""
    import threading
    rng = np.random.default_rng(S.SEED_BASE + 3)
    sc = S.draw_scene(rng, 300_000)
    base = S.draw_base(rng, sc.K, 1)
    mlp = S.draw_mlp(rng, 1)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rxgs.Context()
    h = ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), d(base),
                         d(S.flatten_mlp(mlp, 1)), C=1)
    budget = 16 << 30
    ctx.serve_start(h, kind=rxgs.OUT_RSSI, max_batch_receivers=2048, max_batch_views=16,
                    mem_budget=budget, slots=2)

    def run(dur, rate_hz):
        reqs = S.serve_requests(rng, max(1, int(dur * rate_hz)), rate_hz)
        done = []
        tickets = []
        lock = threading.Lock()

        def poller():
            i = 0
            while True:
                with lock:
                    if i < len(tickets):
                        tk, n = tickets[i]
                    elif len(tickets) == len(reqs):
                        return
                    else:
                        tk = None
                if tk is None:
                    time.sleep(0.0005)
                    continue
                ctx.serve_poll(tk, n, timeout_us=-1)
                done.append(time.perf_counter())
                i += 1

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if r["t"] > now:
                time.sleep(r["t"] - now)
            tk = ctx.serve_submit(r["tx"], r["rx"])
            with lock:
                tickets.append((tk, r["rx"].shape[0]))
        th.join()
        wall = time.perf_counter() - t0
        return len(reqs), sum(r["rx"].shape[0] for r in reqs), wall

    run(warm, rate)                      # plans and graphs for the size classes
    ctx.serve_reset_stats()
    nreq, nrx, wall = run(seconds, rate)
    st = ctx.serve_stats()
    # the same stream at 0.5x, 2x and 4x the rate (shorter runs)
    sweep = []
    for f in sweep_factors:
        ctx.serve_reset_stats()
        n2, r2, w2 = run(sweep_seconds, rate * f)
        s2 = ctx.serve_stats()
        sweep.append({"offered_rps": rate * f, "achieved_rps": round(n2 / w2, 2),
                      "receivers_per_s": round(r2 / w2, 1), "requests": n2,
                      "p50_ms": s2["p50_ms"], "p99_ms": s2["p99_ms"], "max_ms": s2["max_ms"],
                      "mean_batch_receivers": s2["mean_batch_receivers"],
                      "plans_built": s2["plans_built"]})
    ctx.serve_stop()
    ctx.close()
    return {"seconds": seconds, "offered_rps": rate, "achieved_rps": round(nreq / wall, 2),
            "receivers_per_s": round(nrx / wall, 1), "requests": nreq,
            "p50_ms": st["p50_ms"], "p90_ms": st["p90_ms"], "p99_ms": st["p99_ms"],
            "max_ms": st["max_ms"], "batches": st["batches"],
            "mean_batch_receivers": st["mean_batch_receivers"], "failed": st["failed"],
            "retried": st["retried"], "plans_built": st["plans_built"],
            "mem_budget_bytes": budget, "slots": 2, "rate_sweep": sweep,
            "workload": "300k Gaussians, MLP radiance, RSSI, Poisson arrivals, n log-uniform 1..1024"}


def batched_csi_bench(torch, rxgs, S, reps=3):
    """300,000 Gaussians, 256 receivers in batches of U{1..64} (one
    transmitter each), CSI over 52 subcarriers from the bf16 MLP, one
    persistent render launch per batch set under a CUDA graph."""
    w = S.workload_csi()
    sc, C = w["scene"], w["C"]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rxgs.Context()
    h = ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), d(w["base"]),
                         d(S.flatten_mlp(w["mlp"], C)), C=C, bf16=True)
    R = int(sum(w["sizes"]))
    csi = torch.empty((R, C, 2), device="cuda")
    tx, rx = d(w["tx"]), d(w["rx"])
    ctx.render_batched(h, tx, rx, w["sizes"], rxgs.OUT_CSI, csi=csi)   # plan + graph capture
    ctx.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ctx.render_batched(h, tx, rx, w["sizes"], rxgs.OUT_CSI, csi=csi)
    b.record()
    ctx.sync()
    ms = a.elapsed_time(b) / reps
    ctx.close()
    return {"receivers": R, "batches": len(w["sizes"]), "subcarriers": C,
            "ms_per_call": round(ms, 3), "csi_per_s": round(R / (ms / 1e3), 1),
            "workload": "300k Gaussians, 256 rx in U{1..64} batches, C=52, bf16 MLP, CSI"}


def coverage_bench(torch, rxgs, S, reps=3, K=None):
    """Coverage map: 1,000,000 Gaussians, 16 transmitters x 1,024 receivers,
    180x360 grid, explicit radiance [1024, 1M, 1, 2] (8.2 GB, resident).
    One step = the transmitter-side preparation of the 16 views (projection,
    key emission, radix sort, tile ranges), RSSI through the visibility path,
    and the backward from an RSSI cotangent to radiance and opacity (the
    radiance gradient is another 8.2 GB), timed as a whole with CUDA events.
    Roofline: HBM, for the weighted sum (the radiance read once for all 16
    views) and the visibility backward (the radiance read once more, the
    gradient read and written once)."""
    w = (S.workload_coverage(with_radiance=False) if K is None
         else S.workload_coverage(K=K, with_radiance=False))
    g, sc = w["grid"], w["scene"]
    M, N, K = w["tx"].shape[0], w["rx"].shape[0], sc.K
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rxgs.Context(H=g.H, W=g.W, theta0_deg=g.theta0_deg)
    h = ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), None, None, C=1)
    rad = S.hashed_radiance_torch(torch, N, K, "cuda")
    txd = d(w["tx"])
    rssi = torch.empty((M, N), device="cuda")
    csi = torch.empty((M, N, 1, 2), device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(S.SEED_BASE + 41)
    grssi = torch.randn((M, N), device="cuda", generator=gen)
    d_rad = torch.zeros((N, K, 1, 2), device="cuda")
    d_tau = torch.zeros(K, device="cuda")

    def step():
        views = ctx.prepare(h, txd)
        ctx.render_views(views, None, N, rxgs.OUT_RSSI | rxgs.OUT_CSI, radiance=rad, rssi=rssi,
                         csi=csi, reduce_path=1)
        ctx.render_backward(views, None, N, rxgs.OUT_RSSI, radiance=rad, grad_rssi=grssi,
                            fwd_csi=csi, grad_radiance=d_rad, grad_opacity=d_tau)
        ctx.release_views(views)

    for _ in range(2):
        step()
    ctx.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    a.record()
    for _ in range(reps):
        step()
    b.record()
    ctx.sync()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ctx.close()
    ms = a.elapsed_time(b) / reps
    stages = {k: round(v["ms"] / reps, 3) for k, v in prof["stages"].items()}
    pk, src = peaks()
    rad_bytes = 8.0 * N * K

    def hbm(stage, nbytes, what):
        if stage not in prof["stages"]:
            return None
        kms = prof["stages"][stage]["ms"] / prof["stages"][stage]["calls"]
        ach = nbytes / (kms / 1e3) / 1e9
        return {"kernel": stage, "bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4), "launch_ms": round(kms, 4),
                "units": what, "peak_source": f"hbm_gbs ({src})"}

    return {"pairs": M * N, "ms_per_step": round(ms, 3), "rssi_per_s": round(M * N / (ms / 1e3), 1),
            "stages_ms_per_step": stages,
            "roofline": [hbm("weighted_sum", rad_bytes, f"radiance [1024, {K:,}, 1, 2] read once"),
                         hbm("vis_bwd", 3 * rad_bytes,
                             "radiance read once, radiance gradient read and written once")],
            "step": "prepare (16 views) + RSSI forward (visibility path) + RSSI backward to "
                    "radiance and opacity",
            "workload": f"{K:,} Gaussians, 16 tx x 1,024 rx, 180x360, explicit radiance "
                        f"[1024,{K},1,2]"}


def fle_bench(torch, rxgs, S, reps=3, lmax=9, K=None):
    """FLE radiance (App. E.2) at the bench scene's size: 100,000 Gaussians,
    32 transmitters x 64 receivers, degree 9 (L = 100 components; the
    coefficient tensor [64, 100k, 2, 100] is 5.1 GB), 90x360 grid: forward
    spectra, and forward + backward (spectra cotangent) to the coefficients
    and the opacity.  Views prepared once outside the timing."""
    w = S.workload_mlp() if K is None else S.workload_mlp(K=K)
    g, sc = w["grid"], w["scene"]
    M, N, K = w["tx"].shape[0], w["rx"].shape[0], sc.K
    L = (lmax + 1) ** 2
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rxgs.Context(H=g.H, W=g.W)
    h = ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), None, None, C=1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(S.SEED_BASE + 50)
    coeffs = torch.randn((N, K, 2, L), device="cuda", generator=gen) * 0.1
    gspec = torch.randn((M, N, g.H, g.W, 1, 2), device="cuda", generator=gen)
    spec = torch.empty((M, N, g.H, g.W, 1, 2), device="cuda")
    d_fle = torch.zeros_like(coeffs)
    d_tau = torch.zeros(K, device="cuda")
    views = ctx.prepare(h, d(w["tx"]))

    def fwd():
        ctx.render_views(views, None, N, rxgs.OUT_SPECTRA, spectra=spec, fle_coeffs=coeffs,
                         fle_lmax=lmax)

    def fwd_bwd():
        fwd()
        ctx.render_backward(views, None, N, rxgs.OUT_SPECTRA, grad_spectra=gspec,
                            grad_opacity=d_tau, fle_coeffs=coeffs, fle_lmax=lmax, grad_fle=d_fle)

    # the same with the coefficients conditioned by the global FiLM branch
    # (Eq. film, film_apply; App. E.4 sizes: F = 6, d_c = 16, d = 64)
    rng = np.random.default_rng(S.SEED_BASE + 51)
    film_np = S.draw_film(rng, lmax)
    dims = rxgs.film_sizes(film_np)
    film = d(rxgs.pack_film(film_np))
    base = d(S.draw_fle_base(rng, K, lmax))
    rx_d = d(w["rx"])
    d_base = torch.zeros_like(base)
    d_film = torch.zeros_like(film)

    def film_fwd():
        ctx.render_views(views, rx_d, N, rxgs.OUT_SPECTRA, spectra=spec, fle_lmax=lmax,
                         fle_base=base, film=film, film_dims=dims)

    def film_fwd_bwd():
        film_fwd()
        ctx.render_backward(views, rx_d, N, rxgs.OUT_SPECTRA, grad_spectra=gspec,
                            grad_opacity=d_tau, fle_lmax=lmax, fle_base=base, film=film,
                            film_dims=dims, grad_fle_base=d_base, grad_film=d_film)

    fwd_bwd()
    film_fwd_bwd()
    ctx.sync()
    out = {}
    for name, fn in (("forward", fwd), ("forward_backward", fwd_bwd),
                     ("film_forward", film_fwd), ("film_forward_backward", film_fwd_bwd)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.profile(True)
        ctx.profile_read(reset=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        ctx.sync()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        out[name] = {"ms": round(a.elapsed_time(b) / reps, 3),
                     "stages_ms": {k: round(v["ms"] / reps, 3) for k, v in prof["stages"].items()}}
    ctx.release_views(views)
    ctx.close()
    ms = out["forward_backward"]["ms"]
    ms_f = out["film_forward_backward"]["ms"]
    return {"spectra_per_s_fwd_bwd": round(M * N / (ms / 1e3), 1),
            "film_spectra_per_s_fwd_bwd": round(M * N / (ms_f / 1e3), 1), **out,
            "workload": f"{K} Gaussians, 32 tx x 64 rx, FLE degree 9 (L = 100), 90x360, "
                        "spectra; backward to coefficients and opacity; film_*: base "
                        "coefficients [100k, 2, 100] conditioned by the global FiLM branch "
                        "(18 frequency vectors, d_c = 16, d = 64), backward to the base, "
                        "every FiLM parameter and the opacity"}


def train_bench(torch, rxgs, S, reps=3):
    """Stage II training step at the bench scene's size (100k Gaussians,
    32 tx x 64 rx, MLP radiance, 90x360): render, L1 loss on the amplitude
    spectra, backward to phi_base and the MLP, two Adam updates."""
    from paper_2605_24290_gb300.train import Stage2Trainer
    w = S.workload_mlp()
    g, sc, C = w["grid"], w["scene"], w["C"]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rxgs.Context(H=g.H, W=g.W)
    flat = d(S.flatten_mlp(w["mlp"], C))
    h = ctx.upload_scene(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), d(w["base"]),
                         flat, C=C)
    tx, rx = d(w["tx"]), d(w["rx"])
    M, N = tx.shape[0], rx.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(S.SEED_BASE + 60)
    target = torch.rand((M, N, g.H, g.W, C), device="cuda", generator=gen)
    tr = Stage2Trainer(ctx, h, d(sc.opacity), d(w["base"]), flat)
    for _ in range(2):
        tr.step(tx, rx, target)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    losses = [tr.step(tx, rx, target) for _ in range(reps)]
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    ctx.close()
    return {"ms_per_step": round(ms, 3), "spectra_per_s": round(M * N / (ms / 1e3), 1),
            "loss_first_last": [round(float(losses[0]), 6), round(float(losses[-1]), 6)],
            "workload": "100k Gaussians, 32 tx x 64 rx, MLP radiance, L1 on |R| + Adam (phi_base, MLP)"}


def occupancy_bench(torch, rxgs, S, W, reps=3):
    """Occlusion inputs (App. E.5) on the bench scene: building the 128^3
    grid once, and the bench step (prepare + MLP + forward + backward) with
    the 16 probes per (receiver, Gaussian) pair feeding the local MLP."""
    c = W.ctx
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    c.build_occupancy(W.scene, 128)
    b.record()
    torch.cuda.synchronize()
    build_ms = a.elapsed_time(b)
    W.step()
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        W.step()
    b.record()
    torch.cuda.synchronize()
    step_ms = a.elapsed_time(b) / reps
    c.build_occupancy(W.scene, 0)
    return {"grid": 128, "build_ms": round(build_ms, 3), "step_ms": round(step_ms, 3),
            "workload": "bench step with occlusion probes (16 per pair) in the local MLP"}


# ------------------------------------------------------------ CPU oracle
def cpu_sample(budget_s=15.0, steps=None, npx=16384):
    """The oracle on a bounded sample of the same workload: one transmitter,
    one receiver, the forward and backward over a random pixel subset (plus
    the MLP radiance and its backward for that receiver); scaled to spectra
    per second by the sampled fraction of the grid."""
    from oracle import oracle as O
    from paper_2605_24290_gb300 import synthetic as S
    O.build()
    w = S.workload_mlp()
    g, sc = w["grid"], w["scene"]
    rng = np.random.default_rng(1)
    HW = g.H * g.W
    t_tot, frac_tot = 0.0, 0.0
    n_done = 0
    for s in range(10_000):
        if (steps is not None and s >= steps) or (steps is None and t_tot >= budget_s):
            break
        n_done += 1
        pix = rng.choice(HW, size=npx, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        ti, rj = s % w["tx"].shape[0], s % w["rx"].shape[0]
        rad = O.mlp_radiance(w["mlp"], w["rx"][rj:rj + 1], sc.means, w["base"])
        O.render_pixels(g, sc, w["tx"][ti], rad, pix)
        gsp = rng.normal(size=(npx, 1, 1, 2))
        gr, gt = O.backward_pixels(g, sc, w["tx"][ti], rad, pix, gsp)
        O.mlp_backward(w["mlp"], w["rx"][rj:rj + 1], sc.means, w["base"], gr)
        t_tot += time.perf_counter() - t0
        frac_tot += npx / HW
    return {"value": round(frac_tot / t_tot, 4), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{n_done} x (1 tx, 1 rx, {npx} of {HW} pixels) forward+backward incl. MLP; "
                      f"scaled by the pixel fraction",
            "seconds": round(t_tot, 2)}


def reference_bench(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    npx = 4096
    for _ in range(args.warmup):
        cpu_sample(steps=1, npx=npx)
    t0 = time.perf_counter()
    vals = []
    for _ in range(args.steps):
        r = cpu_sample(steps=1, npx=npx)
        vals.append(r)
    wall = time.perf_counter() - t0
    frac = len(vals) * (npx / (90 * 360))
    value = frac / sum(r["seconds"] for r in vals)
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(r["seconds"] for r in vals) / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; indoor-room scene recipe)",
            "config": bench_config(world),
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 2)}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rxgs", choices=["rxgs", "reference"])
    ap.add_argument("--loop-pairs", type=int, default=64)
    ap.add_argument("--no-loop", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tile", type=int, nargs=2, default=None, metavar=("H", "W"),
                    help="fixed tile shape instead of the autotuner's choice")
    ap.add_argument("--cols", type=int, default=0, help="columns per CTA with --tile (0: auto)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-coverage", action="store_true")
    ap.add_argument("--no-fle", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-occupancy", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--coverage-gaussians", type=int, default=None,
                    help="Gaussians of the coverage section (default: 1,000,000; smaller for profiling)")
    ap.add_argument("--fle-gaussians", type=int, default=None,
                    help="Gaussians of the FLE section (default: the bench scene's 100,000)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        reference_bench(args)
    else:
        gpu_bench(args)


if __name__ == "__main__":
    main()
