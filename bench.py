#!/usr/bin/env python3
"""Benchmark: TPC clusters/s tracked on one GB300, batched vs plain, plus the adjoint calibration
gradient cost (arxiv 1712.09434 section 3; Table 1 measures the same batched-vs-plain effect).

One step = the whole hot path over the batched workload (64 events, multiplicity log-uniform in
[100, 20000] tracks, 10 % loopers, 20 % noise, seeds 2000+e): tpc_track_batch (grid, neighbour
finding, chains, following, selection, merge, FP32 Kalman refit; one CUDA graph) followed by
tpc_refit_grad (refit + hand-written adjoint, FP64 reductions) on all tracks of the batch.
value = clusters of the batch / step time.  Inputs are device-resident when the timed region
starts; L2 is flushed (256 MB write) between timed steps.

Also reported: the plain per-event form (tpc_track_event + tpc_refit_grad per event) on the same
events, the adjoint cost per central event with an injected calibration, per-stage times, the
roofline of the dominant stage, the oracle CPU baseline, and an end-to-end number through the
binding with host buffers (H2D of the inputs and D2H of the results inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1712_09434_gb300 import synth  # noqa: E402

METRIC = "TPC clusters/s tracked on 1 GB300, batched vs plain; adjoint calib-grad us/event"
# kernels of one step (one graph): tracking (bin offset check 2, grid 1, links 1, chains 8, follow 2,
# select 1, merge 17, length order of the tracks 3, refit 1) + refit and adjoint of its tracks
# (forward and reverse pass 2, reduce 2; the stored-state form adds the chunk lengths and their
# scan, 4; the hits were packed, the tracks sorted by length and the bin offsets checked by the
# tracking part)
LAUNCHES_TRACKING = 36
LAUNCHES_REFIT_GRAD = {"checkpoints": 4, "stored states": 8}
# copies of the central calibration event whose refit + adjoint run in one call (cost per event
# when the gradient is summed over several events)
CENTRAL_COPIES = 8

def launches_per_step(tuning_best):
    form = "stored states" if tuning_best and tuple(tuning_best.get("refit_grad", (0, 0, 0)))[2] == 1 else "checkpoints"
    return LAUNCHES_TRACKING + LAUNCHES_REFIT_GRAD[form], form
WORKLOAD = "batch-64-events-logU-100-20000-tracks-20pct-noise"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------------

def make_batch(n_events, seed0):
    cache = os.path.join(tempfile.gettempdir(), "tpc_batch_%d_%d.npz" % (n_events, seed0))
    if os.path.exists(cache):
        z = np.load(cache, allow_pickle=False)
        return dict(z)
    t = time.time()
    evs = [synth.make_event(c) for c in synth.batch_configs(n_events=n_events, seed0=seed0)]
    b = synth.concat_events(evs)
    d = dict(pad=b.pad_fp, tim=b.time_fp, bin_off=b.bin_off, ev_off=b.ev_off,
             ev_bin_off=np.stack([e.bin_off for e in evs]))
    tmp = cache[:-4] + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, **d)
    os.replace(tmp, cache)
    log("generated %d events, %d clusters in %.1f s" % (n_events, b.n_clusters, time.time() - t))
    return d


def make_frame(n_events, seed0, per_drift=5.0, slice_len=synth.DRIFT_LSB, seed=3000):
    """The events of the batch overlaid in one continuous readout stream (collision times of a
    Poisson process, per_drift collisions per drift length) and cut into slices of slice_len LSB."""
    cache = os.path.join(tempfile.gettempdir(), "tpc_frame_%d_%d_%g_%d_%d.npz" % (n_events, seed0, per_drift,
                                                                                   slice_len, seed))
    if os.path.exists(cache):
        return dict(np.load(cache, allow_pickle=False))
    d = make_batch(n_events, seed0)
    t = time.time()
    evs = []
    for e in range(n_events):
        a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
        evs.append(types.SimpleNamespace(pad_fp=d["pad"][a:b], time_fp=d["tim"][a:b], bin_off=d["ev_bin_off"][e],
                                         mc_track=np.full(b - a, -1, np.int32), n_clusters=b - a))
    tf = synth.time_frame(evs, per_drift=per_drift, slice_len=slice_len, seed=seed)
    f = dict(pad=tf.pad_fp, tim=tf.time_fp, bin_off=tf.bin_off, n_slices=np.int64(tf.n_slices),
             slice_len=np.int64(tf.slice_len), t0=tf.t0)
    tmp = cache[:-4] + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, **f)
    os.replace(tmp, cache)
    log("time frame: %d collisions, %d slices, %d clusters in %.1f s" % (n_events, tf.n_slices, tf.n_clusters,
                                                                          time.time() - t))
    return f


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "tpc_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception as e:   # no nvidia-smi: report nothing rather than guess
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# native (CUDA) arm
# ---------------------------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp32_peak(seconds=1.0):
    """Measured FP32 FMA throughput of this GPU (tpc_fma_peak): 4 CTAs of 256 threads per SM,
    8 independent FMA chains per thread, one launch of ~`seconds` timed with CUDA events (median of
    three) while nvidia-smi samples the SM clock.  The roof of the Kalman refit and its adjoint."""
    import torch
    from paper_1712_09434_gb300 import capi
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ctas, threads = 4, 256
    out = torch.empty(sms * ctas * threads, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(iters):
        e0.record()
        fl = capi.tpc_fma_peak(out, iters, ctas, threads)
        e1.record()
        e1.synchronize()
        return fl, e0.elapsed_time(e1) * 1e-3

    run(1000)
    fl, t = run(20000)
    iters = max(1000, int(20000 * seconds / max(t, 1e-6)))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    rates = []
    for _ in range(3):
        fl, t = run(iters)
        rates.append(fl / t / 1e12)
    clk = clocks.stop()
    return {"tflops": float(np.median(rates)), "runs": [float(r) for r in rates], "seconds_per_run": t,
            "config": "%d SMs x %d CTAs x %d threads, 8 FMA chains per thread" % (sms, ctas, threads),
            "clocks": clk}


def shard_seed0(rank):
    """First event seed of a rank: weak scaling, every rank tracks its own batch of events with no
    data exchange (events are independent; the seeds of two ranks never overlap for <= 1000 events)."""
    return 2000 + 1000 * rank


def aggregate(ms_local, units_local, world, device="cpu"):
    """Whole-job timing over ranks: the step time is the slowest rank's, the units are the sum over
    ranks; value = units / time.  world == 1 needs no process group."""
    if world <= 1:
        return float(ms_local), int(units_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([int(units_local)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def run_native(args, rank, world):
    import torch
    from paper_1712_09434_gb300 import capi

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    seed0 = shard_seed0(rank)
    d = make_batch(args.events, seed0)
    n_clusters = int(d["pad"].shape[0])
    n_ev = args.events
    cl = capi.Clusters.from_numpy(d["pad"], d["tim"], d["bin_off"], n_ev)
    # track capacity of the outputs: one track per 64 clusters, 2.4 times the 218,673 tracks of the
    # 64-event batch and 1.9 times the 272,526 slice tracks of its time frame (beyond it the library
    # reports CAPACITY, which every timed leg checks).  It sizes the per-track result arrays that the
    # end-to-end leg copies back every step; at one track per 10 clusters (the bound from the 10-hit
    # minimum) they are 585 instead of 316 MB, and the larger host transfers slow the overlapped
    # compute (measured 2.5 against 2.9e9 clusters/s end to end)
    cap_t = n_clusters // 64 + 1024
    ctx = capi.Context(max_clusters=n_clusters, max_events=n_ev)
    tr = capi.Tracks(n_clusters, n_ev, cap_t, n_clusters)
    theta = torch.tensor(synth.theta_nominal(), dtype=torch.float64, device=dev)
    s_chi2 = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(73, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    # calibration track selection (consistent tracks, nominal chi2/ndf < 5), fixed once: the
    # tracks of a step are identical every step (the tracking is deterministic)
    ctx.tpc_track_batch(cl, tr)
    torch.cuda.synchronize()

    def select(t, n):
        ok = (t.ndf[:n] > 0) & (t.chi2[:n] < 5.0 * t.ndf[:n].float())
        return ok.float().contiguous()

    w_batch = select(tr, int(tr.n_tracks.item()))

    def step():       # tracking + refit / adjoint of the tracks: one CUDA graph launch
        ctx.tpc_track_refit_batch(cl, tr, theta, s_chi2, grad, w_batch)

    # launch shapes: autotuned on this workload (outside the timed region), or from the cache
    from paper_1712_09434_gb300 import tune
    tkey = tune.workload_key(n_ev, n_clusters)
    tuning_info = {"key": tkey, "source": "library defaults"}
    if args.only_step or args.no_autotune:
        cached = tune.load(tkey)
        if cached:
            ctx.tpc_set_tuning(tune.to_struct({k: tuple(v) for k, v in cached["best"].items()}))
            tuning_info.update(source="cache", best=cached["best"])
    else:
        t_tune = time.time()
        best, rep = tune.autotune(ctx, step, log=log if rank == 0 else None)
        d_ms, t_ms = rep["default_stage_ms"], rep["tuned_stage_ms"]
        tuning_info.update(source="autotuned in this run", seconds=time.time() - t_tune,
                           best={k: list(v) for k, v in best.items()},
                           default_ms=sum(d_ms.values()), tuned_ms=sum(t_ms.values()))
        if args.store_tuning and rank == 0:
            tune.store(tkey, {"best": tuning_info["best"], "report": rep}, path=args.store_tuning)

    def timed(fn, k, w, profile=False):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        st = ctx.tpc_sync_status()
        if st != 0:
            raise RuntimeError("device status %d" % st)
        if profile:
            ctx.tpc_profile_enable(True)
            ctx.tpc_profile_read(reset=True)
        total = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(k):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if profile:
                ctx.tpc_profile_read()
        prof = None
        if profile:
            prof = ctx.tpc_profile_read(reset=True)
            ctx.tpc_profile_enable(False)
        return total / k, prof

    # Two batches in flight: a second context with its own device copy of the inputs and its own
    # outputs runs every other step on a second stream, so the latency-bound stages of one batch
    # overlap those of the other (a context's calls stay ordered on its own stream).
    ctx2 = capi.Context(max_clusters=n_clusters, max_events=n_ev)
    if tuning_info.get("best"):
        ctx2.tpc_set_tuning(tune.to_struct({k: tuple(v) for k, v in tuning_info["best"].items()}))
    cl2 = capi.Clusters(cl.pad_fp.clone(), cl.time_fp.clone(), cl.bin_off.clone(), n_ev)
    tr2 = capi.Tracks(n_clusters, n_ev, cap_t, n_clusters)
    s_chi2_2, grad_2 = torch.empty_like(s_chi2), torch.empty_like(grad)
    lanes = [(ctx, cl, tr, s_chi2, grad, torch.cuda.Stream()), (ctx2, cl2, tr2, s_chi2_2, grad_2, torch.cuda.Stream())]

    def steps_in_flight(k_steps):
        e_start = torch.cuda.Event()
        e_start.record(stream)
        for c_, cl_, tr_, sc_, gr_, st_ in lanes:
            st_.wait_event(e_start)
        for k in range(k_steps):
            c_, cl_, tr_, sc_, gr_, st_ = lanes[k % 2]
            c_.tpc_track_refit_batch(cl_, tr_, theta, sc_, gr_, w_batch, stream=st_)
        for c_, cl_, tr_, sc_, gr_, st_ in lanes:
            stream.wait_stream(st_)

    steps_in_flight(max(args.warmup, 2))
    torch.cuda.synchronize()
    if ctx.tpc_sync_status() != 0 or ctx2.tpc_sync_status() != 0:
        raise RuntimeError("device status after the warm-up steps")
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps_in_flight(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if ctx.tpc_sync_status() != 0 or ctx2.tpc_sync_status() != 0:
        raise RuntimeError("device status after the timed steps")
    ms_all, n_cl_all = aggregate(ms_step, n_clusters, world, dev)
    # one batch at a time on one stream, L2 flushed before every step
    ms_single, _ = timed(step, max(3, min(args.steps, 20)), 1)
    ms_single, _ = aggregate(ms_single, n_clusters, world, dev)
    # per-stage times from CUDA events inside the graph, in separate (untimed) steps
    _, prof = timed(step, max(3, min(args.steps, 10)), 1, profile=True)
    st = ctx.tpc_sync_status()
    assert st == 0, st
    res = tr.to_host()
    n_tracks, n_hits = res["n_tracks"], int(res["trk_off"][-1])

    out = {"ms_step": ms_all, "ms_single": ms_single, "n_clusters": n_clusters, "n_clusters_all": n_cl_all,
           "n_tracks": n_tracks,
           "n_hits": n_hits, "clocks": clk, "tuning": tuning_info, "prof": prof}
    if args.only_step:
        return out
    # the measured FP32 roof of the Kalman stages (seconds-long FMA loop, clocks sampled)
    out["fp32_peak"] = fp32_peak()

    # end to end through the binding with host (pinned) buffers: every step copies its inputs in
    # and the whole result set out (all outputs of tpc_track_batch, sum of chi2 and gradient)
    h_pad = torch.from_numpy(d["pad"]).pin_memory()
    h_tim = torch.from_numpy(d["tim"].view(np.int16)).pin_memory()
    h_bo = torch.from_numpy(d["bin_off"]).pin_memory()
    d_pad, d_tim, d_bo = cl.pad_fp, cl.time_fp, cl.bin_off

    def out_views(t_):
        return (t_.label[:n_clusters], t_.trk_off[:cap_t + 1], t_.trk_hits[:n_clusters], t_.ev_trk_off[:n_ev + 1],
                t_.par[:cap_t * 5], t_.xref[:cap_t], t_.cov[:cap_t * 15], t_.chi2[:cap_t], t_.ndf[:cap_t],
                t_.n_tracks[:1])

    def host_set():
        return tuple(torch.empty_like(x, device="cpu").pin_memory() for x in out_views(tr)) + \
            (torch.empty(74, dtype=torch.float64).pin_memory(),)

    h_seq = host_set()

    def e2e():
        d_pad.copy_(h_pad, non_blocking=True)
        d_tim.copy_(h_tim, non_blocking=True)
        d_bo.copy_(h_bo, non_blocking=True)
        step()
        for dst, src in zip(h_seq, out_views(tr)):
            dst.copy_(src, non_blocking=True)
        h_seq[-1][:1].copy_(s_chi2, non_blocking=True)
        h_seq[-1][1:].copy_(grad, non_blocking=True)

    if world > 1:
        torch.distributed.barrier()
    ms_e2e_seq, _ = timed(e2e, max(1, min(args.steps, 5)), 1)
    ms_e2e_seq, _ = aggregate(ms_e2e_seq, n_clusters, world, dev)
    h2d = h_pad.numel() * 2 + h_tim.numel() * 2 + h_bo.numel() * 4
    d2h = sum(x.numel() * x.element_size() for x in h_seq)
    # the device-resident result of this step, for the check of every host copy below
    ref_red = torch.cat([s_chi2, grad]).cpu()

    # pipelined: the two contexts of the timed steps take the steps in turn, each on its own compute
    # stream.  Every context has two buffer sets, inputs and outputs, used by its steps in turn: a
    # step's inputs are copied in while the context's previous step (on the other set) computes, and
    # its results go to the host on a copy stream straight from the output buffers while the next
    # steps compute; a set is reused only after its results reached the host.  No context waits for a
    # host transfer, and no device copy of the results is made.
    # one input and one result copy stream per context, so that one context's copies never queue
    # behind the other's
    s_ins = [torch.cuda.Stream(), torch.cuda.Stream()]
    s_outs = [torch.cuda.Stream(), torch.cuda.Stream()]
    s_out = s_outs[0]

    def dev_inputs():
        return capi.Clusters(torch.empty_like(d_pad), torch.empty_like(d_tim), torch.empty_like(d_bo), n_ev)

    cls = [[cl, dev_inputs()], [cl2, dev_inputs()]]
    trs = [[tr, capi.Tracks(n_clusters, n_ev, cap_t, n_clusters)],
           [tr2, capi.Tracks(n_clusters, n_ev, cap_t, n_clusters)]]
    reds = [[(s_chi2, grad), (torch.empty_like(s_chi2), torch.empty_like(grad))],
            [(s_chi2_2, grad_2), (torch.empty_like(s_chi2), torch.empty_like(grad))]]
    h_outs = [[h_seq, host_set()], [host_set(), host_set()]]
    ev_in = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]
    ev_comp = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]
    ev_out = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]

    def e2e_pipelined(n_steps, first=0):
        for k in range(first, first + n_steps):
            b, j = k % 2, (k // 2) % 2                    # context, buffer set of this context
            c, t_, (sc, gr) = cls[b][j], trs[b][j], reds[b][j]
            ho = h_outs[b][j]
            cx, cs = lanes[b][0], lanes[b][5]
            s_in, s_out = s_ins[b], s_outs[b]
            with torch.cuda.stream(s_in):                 # inputs (free once this set's last step ran)
                s_in.wait_event(ev_comp[b][j])
                c.pad_fp.copy_(h_pad, non_blocking=True)
                c.time_fp.copy_(h_tim, non_blocking=True)
                c.bin_off.copy_(h_bo, non_blocking=True)
                ev_in[b][j].record(s_in)
            cs.wait_event(ev_in[b][j])
            cs.wait_event(ev_out[b][j])                   # this set's last results are on the host
            cx.tpc_track_refit_batch(c, t_, theta, sc, gr, w_batch, stream=cs)
            ev_comp[b][j].record(cs)
            with torch.cuda.stream(s_out):                # results to the host
                s_out.wait_event(ev_comp[b][j])
                for dst, src in zip(ho[:-1], out_views(t_)):
                    dst.copy_(src, non_blocking=True)
                ho[-1][:1].copy_(sc, non_blocking=True)
                ho[-1][1:].copy_(gr, non_blocking=True)
                ev_out[b][j].record(s_out)
        for s_ in s_ins + s_outs:
            stream.wait_stream(s_)
        for lane_ in lanes:
            stream.wait_stream(lane_[5])

    n_pipe = max(8, min(args.steps, 40))
    e2e_pipelined(4)                       # warm: every buffer set of both contexts captured once
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    # three timed windows of n_pipe steps each; the line reports their median and lists all three
    ms_windows = []
    for w_ in range(3):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in [lane_[5] for lane_ in lanes] + s_ins + s_outs:
            s_.wait_event(e0)
        e2e_pipelined(n_pipe, first=4 + 4 * n_pipe * w_)
        e1.record(stream)
        e1.synchronize()
        ms_windows.append(e0.elapsed_time(e1) / n_pipe)
    ms_e2e = float(np.median(ms_windows))
    assert ctx.tpc_sync_status() == 0 and ctx2.tpc_sync_status() == 0
    ms_e2e, _ = aggregate(ms_e2e, n_clusters, world, dev)
    # every host result set (both contexts, both buffer sets: the last steps of the timed loop) must
    # equal the device-resident result bit for bit; a race between a host copy and the next step
    # writing the same output set would show here
    torch.cuda.synchronize()
    nt, nh = res["n_tracks"], int(res["trk_off"][-1])
    want = (res["label"][:n_clusters], res["trk_off"], res["trk_hits"], res["ev_trk_off"][:n_ev + 1],
            res["par"].reshape(-1), res["xref"], res["cov"].reshape(-1), res["chi2"], res["ndf"],
            np.array([nt], np.int32))
    prefix = (n_clusters, nt + 1, nh, n_ev + 1, 5 * nt, nt, 15 * nt, nt, nt, 1)
    e2e_checked = 0
    for b in range(2):
        for j in range(2):
            ho = h_outs[b][j]
            for k, (got, w_, m) in enumerate(zip(ho[:-1], want, prefix)):
                if not np.array_equal(got[:m].numpy(), np.asarray(w_)[:m]):
                    raise RuntimeError("end-to-end result %d of context %d, set %d differs from the device result"
                                       % (k, b, j))
            if not torch.equal(ho[-1], ref_red):
                raise RuntimeError("end-to-end sum of chi2 / gradient of context %d, set %d differs" % (b, j))
            e2e_checked += 1

    # the host link alone: one step's input copies, and one step's result copies, with no compute
    def copies(direction):
        with torch.cuda.stream(s_out):
            for _ in range(5):
                if direction == "h2d":
                    d_pad.copy_(h_pad, non_blocking=True)
                    d_tim.copy_(h_tim, non_blocking=True)
                    d_bo.copy_(h_bo, non_blocking=True)
                else:
                    for dst, src in zip(h_outs[1][1][:-1], out_views(tr)):
                        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(s_out)
        with torch.cuda.stream(s_out):
            for _ in range(10):
                if direction == "h2d":
                    d_pad.copy_(h_pad, non_blocking=True)
                    d_tim.copy_(h_tim, non_blocking=True)
                    d_bo.copy_(h_bo, non_blocking=True)
                else:
                    for dst, src in zip(h_outs[1][1][:-1], out_views(tr)):
                        dst.copy_(src, non_blocking=True)
        c1.record(s_out)
        c1.synchronize()
        return c0.elapsed_time(c1) / 10

    link_ms = {"h2d_ms_per_step": copies("h2d"), "d2h_ms_per_step": copies("d2h")}
    out.update(ms_e2e=ms_e2e, ms_e2e_seq=ms_e2e_seq, h2d=h2d, d2h=d2h, e2e_checked=e2e_checked, link_ms=link_ms,
               e2e_windows=[n_cl_all / (m * 1e-3) for m in ms_windows])
    if rank != 0:
        return out

    # units for the algorithmic byte counts (outside the timed region)
    nc_t = torch.empty(1, dtype=torch.int32, device=dev)
    ctx.tpc_debug_copy(2, nc_t)
    n_chains = int(nc_t.item())
    cn = torch.empty(max(n_chains, 1), dtype=torch.int32, device=dev)
    ctx.tpc_debug_copy(5, cn)
    cand_hits = int(cn[:n_chains].sum().item())
    lens = torch.tensor(np.diff(res["trk_off"]), dtype=torch.float32, device=dev)
    weighted_hits = int((lens * w_batch[:lens.numel()]).sum().item())

    # plain per-event form on the same events
    evs_cl = []
    for e in range(n_ev):
        a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
        evs_cl.append(capi.Clusters.from_numpy(d["pad"][a:b], d["tim"][a:b], d["ev_bin_off"][e], 1))
    tr1 = capi.Tracks(n_clusters, 1, cap_t, n_clusters)
    w_ev = []
    for c in evs_cl:
        ctx.tpc_track_event(c, tr1)
        torch.cuda.synchronize()
        w_ev.append(select(tr1, int(tr1.n_tracks.item())))

    def plain():
        for c, w in zip(evs_cl, w_ev):
            ctx.tpc_track_event(c, tr1)
            ctx.tpc_refit_grad(c, tr1, theta, s_chi2, grad, w)

    ms_plain, _ = timed(plain, max(1, min(args.steps, 5)), 1)

    # continuous readout: the same collisions overlaid in one readout stream at Poisson times (5 per
    # drift length), cut into slices of one drift length, tracked as one batch of slices and
    # joined by the slice merge
    fr = make_frame(n_ev, seed0)
    ns_f, L = int(fr["n_slices"]), int(fr["slice_len"])
    cf = capi.Clusters.from_numpy(fr["pad"], fr["tim"], fr["bin_off"], ns_f)
    tf_s = capi.Tracks(n_clusters, ns_f, cap_t, n_clusters)
    tf_f = capi.Tracks(n_clusters, 1, cap_t, n_clusters)

    def frame_step():
        ctx.tpc_track_batch(cf, tf_s)
        ctx.tpc_merge_slices(cf, tf_s, L, tf_f)

    ms_frame, _ = timed(frame_step, max(3, min(args.steps, 10)), 3)
    ms_fmerge, _ = timed(lambda: ctx.tpc_merge_slices(cf, tf_s, L, tf_f), 10, 3)
    hs, hf = tf_s.to_host(), tf_f.to_host()
    nxt = torch.empty(max(hs["n_tracks"], 1), dtype=torch.int32, device=dev)
    ctx.tpc_debug_copy(9, nxt)
    frame_out = {"value": n_clusters / (ms_frame * 1e-3), "unit": "clusters/s", "ms_per_frame": ms_frame,
                 "slice_merge_ms": ms_fmerge, "collisions": n_ev, "collisions_per_drift_length": 5.0,
                 "slices": ns_f, "slice_len_lsb": L, "clusters": int(fr["pad"].shape[0]),
                 "slice_tracks": hs["n_tracks"], "links": int((nxt[:hs["n_tracks"]] >= 0).sum().item()),
                 "frame_tracks": hf["n_tracks"],
                 "step": "tpc_track_batch over the slices (CUDA graph) + tpc_merge_slices"}
    del tf_s, tf_f, cf

    # the single-event numbers below are other workloads: library default launch shapes
    ctx.tpc_set_tuning(None)

    # adjoint cost on a central event with an injected calibration
    ev5 = synth.make_event(synth.calib_event())
    c5 = capi.Clusters.from_numpy(ev5.pad_fp, ev5.time_fp, ev5.bin_off, 1)
    t5 = capi.Tracks(ev5.n_clusters, 1, ev5.n_clusters // 8 + 1024, ev5.n_clusters)
    ctx.tpc_track_event(c5, t5)
    torch.cuda.synchronize()
    w5 = select(t5, int(t5.n_tracks.item()))
    # references at the vertex from the TPC-ITS matching (inner-tracker tracks with 95 % efficiency
    # and 2 % fakes, generated from the event's particles)
    its5, its_part = synth.its_tracks(ev5)
    its5_d = torch.tensor(its5.astype(np.float32), device=dev)
    nt5 = int(t5.n_tracks.item())
    m_trk = torch.empty(nt5, dtype=torch.int32, device=dev)
    m_its = torch.empty(its5.shape[0], dtype=torch.int32, device=dev)
    a5 = torch.zeros((nt5, 8), dtype=torch.float32, device=dev)
    ms_match, _ = timed(lambda: ctx.tpc_its_match(c5, t5, its5_d, m_trk, m_its, a5), 10, 3)
    ref5 = a5.cpu().numpy().astype(np.float64)
    h5 = t5.to_host()
    mt5 = m_trk.cpu().numpy()
    lead5 = np.array([np.bincount(np.maximum(ev5.mc_track[h5["trk_hits"][a:b]], 0)).argmax()
                      for a, b in zip(h5["trk_off"][:-1], h5["trk_off"][1:])])
    mm = mt5 >= 0
    match_out = {"ms_per_event": ms_match, "tracks": nt5, "its_tracks": int(its5.shape[0]),
                 "matched": int(mm.sum()), "right_particle": float((its_part[mt5[mm]] == lead5[mm]).mean()),
                 "to_fakes": int((its_part[mt5[mm]] < 0).sum()), "with_references": int((ref5[:, 0] > 0).sum())}
    # looper legs of the same event: pairs, their truth, and the loopers whose two legs were found
    pair5 = torch.empty(nt5, dtype=torch.int32, device=dev)
    leg5 = torch.empty(nt5, dtype=torch.int32, device=dev)
    ms_loop, _ = timed(lambda: ctx.tpc_looper_pairs(c5, t5, pair5, leg5), 10, 3)
    p5 = pair5.cpu().numpy()
    pm = p5 >= 0
    kB = abs(synth.KB)
    s_med = np.array([np.nanmedian(ev5.true_s[h5["trk_hits"][a:b]]) if b > a else np.nan
                      for a, b in zip(h5["trk_off"][:-1], h5["trk_off"][1:])])
    half = np.pi * ev5.trk_pt[lead5] / kB            # path length of the far point of each track's particle
    loops = (2 * ev5.trk_pt / kB < synth.R_OUT)      # particles whose circle stays inside the TPC
    out_leg = loops[lead5] & (s_med < half)
    ret_leg = loops[lead5] & (s_med >= half)
    both = np.intersect1d(lead5[out_leg], lead5[ret_leg])
    joined = np.unique(lead5[pm & (lead5 == lead5[np.maximum(p5, 0)])])
    loop_out = {"ms_per_event": ms_loop, "pairs": int(pm.sum() // 2),
                "same_particle": float((lead5[pm] == lead5[p5[pm]]).mean()) if pm.any() else None,
                "loopers_with_both_legs_found": int(both.size),
                "of_them_joined": float(np.isin(both, joined).mean()) if both.size else None}
    th5 = torch.tensor(synth.calib_theta(1005), dtype=torch.float64, device=dev)
    # the adjoint as specified: per-row Kalman states recomputed in the reverse sweep from checkpoints
    # (every 16 steps); then the variant that stores every step's input state (80 B per hit)
    from paper_1712_09434_gb300 import tune as _tune
    ms_grad, _ = timed(lambda: ctx.tpc_refit_grad(c5, t5, th5, s_chi2, grad, w5, a5, 1), 10, 3)
    g_ck = grad.clone()
    ctx.tpc_set_tuning(_tune.to_struct({"refit_grad": (0, 0, 1)}))
    ms_grad_stored, _ = timed(lambda: ctx.tpc_refit_grad(c5, t5, th5, s_chi2, grad, w5, a5, 1), 10, 3)
    ctx.tpc_set_tuning(None)
    assert torch.equal(g_ck, grad), "the two adjoint forms must give identical gradients"
    # the same refit + adjoint over K copies of the event tracked as one batch, in one call: the
    # cost per event when the calibration sums its gradient over several events (one event alone
    # fills about one warp per SM sub-partition, so its time is the latency of its longest tracks)
    K = CENTRAL_COPIES
    bK = synth.concat_events([ev5] * K)
    cK = capi.Clusters.from_numpy(bK.pad_fp, bK.time_fp, bK.bin_off, K)
    tK = capi.Tracks(bK.n_clusters, K, K * (ev5.n_clusters // 8 + 1024), bK.n_clusters)
    ctx.tpc_track_batch(cK, tK)
    hK = tK.to_host()
    assert hK["n_tracks"] == K * nt5 and np.array_equal(
        hK["trk_hits"], np.concatenate([h5["trk_hits"] + e * ev5.n_clusters for e in range(K)])), \
        "the copies must give the event's tracks"
    wK, aK = w5.repeat(K), a5.repeat(K, 1)
    gK = torch.empty_like(grad)
    ms_grad_K, _ = timed(lambda: ctx.tpc_refit_grad(cK, tK, th5, s_chi2, gK, wK, aK, 1), 10, 3)
    assert torch.allclose(gK, K * g_ck, rtol=1e-9, atol=1e-9 * float(g_ck.abs().max())), \
        "K copies must give K times the event's gradient"
    ctx.tpc_set_tuning(_tune.to_struct({"refit_grad": (0, 0, 1)}))
    ms_grad_K_stored, _ = timed(lambda: ctx.tpc_refit_grad(cK, tK, th5, s_chi2, gK, wK, aK, 1), 10, 3)
    ctx.tpc_set_tuning(None)
    del cK, tK, bK

    # plain per-event tracking of single events: the central event above and a 5,000-track event
    single = {}
    ev2 = synth.make_event(synth.full_event())
    c2 = capi.Clusters.from_numpy(ev2.pad_fp, ev2.time_fp, ev2.bin_off, 1)
    t2 = capi.Tracks(ev2.n_clusters, 1, ev2.n_clusters // 8 + 1024, ev2.n_clusters)
    for name, cc, tt, ncl in [("full_event_5000_tracks", c2, t2, ev2.n_clusters),
                              ("central_20000_tracks", c5, t5, ev5.n_clusters)]:
        ms_ev, _ = timed(lambda: ctx.tpc_track_event(cc, tt), 10, 3)
        single[name] = {"clusters": int(ncl), "ms": ms_ev, "clusters_per_s": ncl / (ms_ev * 1e-3)}

    # rules for inefficient data (links across an empty row, gap merge inside a sector) on the
    # central-shaped event with dead rows 60-61, 100-111 and 5 % of the crossings dropped
    evi = synth.make_event(synth.inefficient_central())
    ci = capi.Clusters.from_numpy(evi.pad_fp, evi.time_fp, evi.bin_off, 1)
    ti = capi.Tracks(evi.n_clusters, 1, evi.n_clusters // 10 + 1024, evi.n_clusters)
    rules_out = {"event": "central-shaped, 20000 tracks, dead rows 60-61 and 100-111, 5 % of crossings dropped",
                 "clusters": int(evi.n_clusters)}
    for name, rules in (("plain", 0), ("rules", capi.TPC_RULE_SKIP_ROW | capi.TPC_RULE_GAP_MERGE)):
        ctx.tpc_set_rules(rules)
        ms_r, _ = timed(lambda: ctx.tpc_track_event(ci, ti), 5, 2)
        hi = ti.to_host()
        eff, n_part, fake = synth.track_quality(evi, hi["trk_off"], hi["trk_hits"])
        rules_out[name] = {"ms": ms_r, "tracks": hi["n_tracks"], "found_whole_efficiency": eff, "particles": n_part,
                           "fake_fraction": fake}
    ctx.tpc_set_rules(0)
    del ci, ti

    # calibration recovery: 20 preconditioned gradient steps from the nominal theta
    from paper_1712_09434_gb300 import calib
    t_cal = time.time()
    cres, n_drop, n_calls = calib.calibrate(ctx, c5, t5, w5, ref5, synth.theta_nominal(), steps=20)
    t_cal = time.time() - t_cal
    th_star = synth.calib_theta(1005)
    blocks = (slice(0, 1), slice(1, 37), slice(37, 73))
    rem = [float(np.linalg.norm(cres.theta[b] - th_star[b]) / np.linalg.norm(synth.theta_nominal()[b] - th_star[b]))
           for b in blocks]
    pull = np.abs(cres.theta - th_star) / cres.sigma
    calib_out = {"steps": 20, "gradient_calls": n_calls, "references_dropped": n_drop, "wall_s": t_cal,
                 "objective": "-2 log L: raw errors through the transformation + references at the vertex "
                              "from the TPC-ITS matching",
                 "remaining_distortion_per_block": dict(zip(["s_vd", "d_k", "a_k"], rem)),
                 "max_pull_per_block": dict(zip(["s_vd", "d_k", "a_k"], [float(pull[b].max()) for b in blocks])),
                 "sum_chi2_start_end": [cres.history[0][1], cres.history[-1][1]],
                 "tracks_with_reference": int((ref5[:, 0] > 0).sum())}

    out.update(ms_plain=ms_plain, ms_grad_event=ms_grad, ms_grad_event_stored=ms_grad_stored,
               ms_grad_copies=ms_grad_K, ms_grad_copies_stored=ms_grad_K_stored, its_match=match_out, loopers=loop_out,
               inefficient=rules_out,
               n_tracks_c5=int(t5.n_tracks.item()), prof=prof,
               weighted_hits=weighted_hits,
               calib=calib_out, single=single, frame=frame_out,
               n_chains=n_chains, cand_hits=cand_hits)
    ctx.close()
    return out


# floating-point operations per hit of the Kalman kernels, counted exactly from csrc/kf.cuh by
# tests/kf_flop_count.cpp (a fused multiply-add counts two): the gradient kernel runs the forward
# step once (storing every step's input state) and its adjoint once; the tracking refit runs the
# square-root forward step
FLOP_FWD, FLOP_ADJ, FLOP_SQRT_FWD = 461, 850, 434
# FP32 peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def stage_flops(u, adjoint_form="checkpoints"):
    """FP32 operations of the Kalman stages: the tracking refit runs the square-root forward step per
    hit; the gradient runs the forward step, its adjoint and (checkpoint form) the forward step again
    to recompute the states of each segment."""
    per_hit = FLOP_FWD + FLOP_ADJ + (FLOP_FWD if adjoint_form == "checkpoints" else 0)
    return {"refit": FLOP_SQRT_FWD * u["n_hits"], "refit_grad": per_hit * u["weighted_hits"]}


# algorithmic bytes per stage (compulsory DRAM traffic of each stage's inputs and outputs)
def stage_bytes(u):
    N, C, Hc, T, Ht = u["n_clusters"], u["n_chains"], u["cand_hits"], u["n_tracks"], u["n_hits"]
    return {
        "grid": 10 * N,                 # read (pad, time) 4 B; write packed (Y, Z) 4 B + local index 2 B
        "links": 18 * N,                # read own 4 B + neighbour-row grid 6 B; write up, down 8 B
        "chains": 16 * N + 12 * C,      # read up/down 8 B, write/read chain length 8 B; chain records
        "follow": 8 * Hc + 12 * C,      # candidate hit: slot write 4 B + cluster read 4 B; chain record
        "select": 16 * Hc,              # candidate hit: slot read 4 B, claim 8 B, owner 4 B
        "merge": 12 * Ht + 32 * C,      # track hit: slot read + hit and label write; segment ends
        "refit": 8 * Ht + 92 * T,       # track hit: packed hit 8 B; per track 23 words out
        "pack": 16 * Ht,                # hit index 4 B + cluster 4 B in, packed hit 8 B out
        "refit_grad": 8 * Ht + 104 * T,  # packed hit 8 B; per-track record out
        "reduce": 104 * T,
    }


def finish_native(args, res, world):
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    n_cl_total = res["n_clusters_all"]
    value = n_cl_total / (res["ms_step"] * 1e-3)
    prof, n_calls = res["prof"]
    k = max(n_calls, 1)
    stage_ms = {s: v / k for s, v in prof.items()}
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    byts = stage_bytes(res)
    n_launch, adj_form = launches_per_step(res["tuning"].get("best"))
    flops = stage_flops(res, adj_form)
    fp = res.get("fp32_peak")
    if fp:
        fp32_roof, fp32_kind = fp["tflops"], "measured (tpc_fma_peak, %s)" % fp["config"]
    else:
        fp32_roof, fp32_kind = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    if dom in flops:       # FP32 arithmetic of the Kalman kernels: the FP32 pipe is the roof
        achieved = flops[dom] / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_roof, "unit": "TFLOP/s",
                "frac": achieved / fp32_roof, "peak_kind": fp32_kind, "algorithmic_flops": flops[dom]}
    else:
        achieved = byts[dom] / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_kind": peak_kind, "algorithmic_bytes": byts[dom]}
    plain_value = res["n_clusters"] / (res["ms_plain"] * 1e-3)
    e2e_value = n_cl_total / (res["ms_e2e"] * 1e-3)
    traffic = None
    # DRAM bytes per launch of the dominant kernel from an ncu capture (null if none matches)
    prof_path = os.path.join(ROOT, "profiles", "k_%s_batch64_traffic.json" % dom)
    if os.path.exists(prof_path):
        tj = json.load(open(prof_path))
        if tj.get("stage") == dom and tj.get("workload") == WORKLOAD:
            traffic = tj.get("bytes_per_launch")
    line = {
        "metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32+f32 (f64 reductions)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_events": args.events, "clusters_per_gpu": res["n_clusters"],
                   "tracks_per_gpu": res["n_tracks"],
                   "l2": "not flushed between steps: each step reads its own device copy of the batch (134 MB of "
                         "clusters, above the 129 MB L2) and ~11 GB of workspace; single_stream flushes L2 "
                         "(256 MB write) before every step",
                   "step": "tpc_track_refit_batch: tracking + refit / adjoint of the batch as one CUDA graph "
                           "launch; two batches in flight (two contexts, two streams, steps alternating)"},
        "single_stream": {"value": res["n_clusters_all"] / (res["ms_single"] * 1e-3), "unit": "clusters/s",
                          "ms_per_step": res["ms_single"],
                          "form": "one batch at a time on one stream, L2 flushed before every step"},
        "plain": {"value": plain_value, "unit": "clusters/s", "ms_per_step": res["ms_plain"],
                  "form": "tpc_track_event + tpc_refit_grad per event, same 64 events"},
        "batched_gain": res["n_clusters"] / (res["ms_single"] * 1e-3) / plain_value,
        "adjoint": {"value": res["ms_grad_event"] * 1e3, "unit": "us/event",
                    "event": "central, 20000 tracks, injected calibration, references at the vertex from the "
                             "TPC-ITS matching",
                    "tracks": res["n_tracks_c5"],
                    "form": "refit + adjoint, Kalman states of the reverse sweep recomputed from checkpoints "
                            "every 16 steps",
                    "stored_states": {"value": res["ms_grad_event_stored"] * 1e3, "unit": "us/event",
                                      "form": "variant storing every step's input state (80 B per hit); "
                                              "identical gradient"},
                    "batched": {"value": res["ms_grad_copies"] * 1e3 / CENTRAL_COPIES, "unit": "us/event",
                                "events": CENTRAL_COPIES,
                                "stored_states": res["ms_grad_copies_stored"] * 1e3 / CENTRAL_COPIES,
                                "form": "%d copies of the event tracked as one batch, refit + adjoint of all "
                                        "their tracks in one call (checkpoints; stored_states: the variant); "
                                        "gradient checked to be %d times the event's" % (CENTRAL_COPIES,
                                                                                          CENTRAL_COPIES)}},
        "calibration": res["calib"],
        "its_match": res.get("its_match"),
        "looper_legs": res.get("loopers"),
        "inefficient_data": res.get("inefficient"),
        "single_event": res["single"],
        "time_frame": res["frame"],
        "stage_ms": stage_ms,
        "tuning": res["tuning"],
        "stage_algorithmic_gbs": {k: byts[k] / (stage_ms[k] * 1e-3) / 1e9 for k in stage_ms if k in byts and stage_ms[k] > 0},
        "units": {"clusters": res["n_clusters"], "chains": res["n_chains"], "candidate_hits": res["cand_hits"],
                  "tracks": res["n_tracks"], "track_hits": res["n_hits"], "weighted_track_hits": res["weighted_hits"]},
        "roofline": dict(roof, traffic=traffic),
        "stage_tflops": {k: flops[k] / (stage_ms[k] * 1e-3) / 1e12 for k in flops if stage_ms.get(k, 0) > 0},
        "stage_fp32_frac": {k: flops[k] / (stage_ms[k] * 1e-3) / 1e12 / fp32_roof for k in flops
                            if stage_ms.get(k, 0) > 0},
        "fp32_peak": fp if fp else {"tflops": FP32_PEAK_TFLOPS, "kind": fp32_kind},
        "adjoint_form_in_step": adj_form,
        "e2e": {"value": e2e_value, "unit": "clusters/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"],
                "form": "through the binding from pinned host buffers; two contexts taking the steps in turn, "
                        "two input and output buffer sets per context used in turn; host copies on their "
                        "own streams overlapping the compute; every step copies the whole result set back "
                        "(labels, track offsets and hits, event offsets, parameters, reference x, "
                        "covariances, chi2, ndf, track count, sum of chi2 and gradient)",
                "checked": "%d host result sets equal to the device-resident result bit for bit" %
                           res.get("e2e_checked", 0),
                "sequential_value": n_cl_total / (res["ms_e2e_seq"] * 1e-3),
                "host_link_alone": res.get("link_ms"),
                "windows": res.get("e2e_windows")},
        "gpu_launches": n_launch * args.steps,
        "clocks": res["clocks"],
    }
    return line


# ---------------------------------------------------------------------------------------------
# oracle (CPU) arm
# ---------------------------------------------------------------------------------------------

def oracle_sample(d, max_seconds):
    """Time the FP64 oracle (tracking S2-S7 + refit S8) event by event until max_seconds of work;
    returns (clusters, seconds, events)."""
    from oracle import oracle as O
    n = len(d["ev_off"]) - 1
    done_cl, t_tot, k = 0, 0.0, 0
    for e in range(n):
        a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
        pad, tim, bo = d["pad"][a:b], d["tim"][a:b], d["ev_bin_off"][e]
        t = time.perf_counter()
        r = O.track_event(pad, tim, bo)
        O.fit(pad, tim, bo, r["trk_off"], r["trk_hits"])
        t_tot += time.perf_counter() - t
        done_cl += b - a
        k += 1
        if t_tot >= max_seconds:
            break
    return done_cl, t_tot, k


def _oracle_worker(args):
    """One host process of the parallel oracle run: takes events e = start, start + stride, ...
    (of the cached batch) and tracks + refits each until `seconds` of work; returns (clusters,
    seconds of work)."""
    n_events, seed0, start, stride, seconds = args
    d = make_batch(n_events, seed0)
    from oracle import oracle as O
    O.build()
    done_cl, busy = 0, 0.0
    for e in range(start, n_events, stride):
        a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
        pad, tim, bo = d["pad"][a:b], d["tim"][a:b], d["ev_bin_off"][e]
        t = time.perf_counter()
        r = O.track_event(pad, tim, bo)
        O.fit(pad, tim, bo, r["trk_off"], r["trk_hits"])
        busy += time.perf_counter() - t
        done_cl += b - a
        if busy >= seconds:
            break
    return done_cl, busy


def oracle_parallel(n_events, seed0, seconds, cores=None):
    """The oracle, unchanged, on `cores` host processes (one event per process at a time; events
    are independent): clusters/s = clusters done / the longest busy time of a process."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")            # never fork a process that has touched the GPU
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(n_events, seed0, i, cores, seconds) for i in range(cores)])
    cl = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return cl, t, cores


def cpu_baseline(d, seconds=15.0, n_events=64, seed0=2000):
    from oracle import oracle as O
    O.build()
    cl1, t1, k1 = oracle_sample(d, seconds / 3)
    cl, t, cores = oracle_parallel(n_events, seed0, seconds)
    return {"value": cl / t, "unit": "clusters/s", "cores": cores, "kind": "oracle",
            "sample": "the 64 events spread over %d host processes, each tracking + FP64-refitting its events "
                      "for ~%.0f s (%d clusters done)" % (cores, seconds, cl),
            "single_core": {"value": cl1 / t1, "sample": "first %d events (%d clusters), one process" % (k1, cl1)}}


def run_reference(args, rank, world):
    """The oracle, unchanged, as the reference arm: every step spreads the batch's events over all
    host cores for ~5 s of work per process."""
    if rank != 0:
        return
    import multiprocessing as mp
    make_batch(args.events, 2000)                     # generate / cache once
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    tot_cl, tot_t = 0, 0.0
    with ctx.Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [(args.events, 2000, i, cores, 0.5) for i in range(cores)])
        for k in range(args.steps):
            res = pool.map(_oracle_worker, [(args.events, 2000, (i + k) % cores, cores, 5.0) for i in range(cores)])
            tot_cl += sum(r[0] for r in res)
            tot_t += max(r[1] for r in res)
    value = tot_cl / tot_t
    sample = "the %d events over %d host processes, ~5 s of tracking + FP64 refit per process and step" % (
        args.events, cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_events": args.events},
            "cpu_baseline": {"value": value, "unit": "clusters/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------

def adjoint_event(form, calls=10):
    """Refit + adjoint of the central calibration event (references from the TPC-ITS matching, raw
    errors) in one form, library default launch shapes otherwise: ms per call."""
    import numpy as np
    import torch
    from paper_1712_09434_gb300 import capi, tune
    dev = "cuda"
    ev = synth.make_event(synth.calib_event())
    cl = capi.Clusters.from_numpy(ev.pad_fp, ev.time_fp, ev.bin_off, 1)
    tr = capi.Tracks(ev.n_clusters, 1, ev.n_clusters // 8 + 1024, ev.n_clusters)
    ctx = capi.Context(max_clusters=ev.n_clusters, max_events=1)
    ctx.tpc_track_event(cl, tr)
    h = tr.to_host()
    nt = h["n_tracks"]
    w = torch.tensor(((h["ndf"] > 0) & (h["chi2"] < 5.0 * np.maximum(h["ndf"], 1))).astype(np.float32), device=dev)
    its, _ = synth.its_tracks(ev)
    its_d = torch.tensor(its.astype(np.float32), device=dev)
    m_trk = torch.empty(nt, dtype=torch.int32, device=dev)
    m_its = torch.empty(its.shape[0], dtype=torch.int32, device=dev)
    anchor = torch.zeros((nt, 8), dtype=torch.float32, device=dev)
    ctx.tpc_its_match(cl, tr, its_d, m_trk, m_its, anchor)
    th = torch.tensor(synth.calib_theta(1005), dtype=torch.float64, device=dev)
    s_chi2 = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(1 + 2 * synth.N_SECTORS, dtype=torch.float64, device=dev)
    ctx.tpc_set_tuning(tune.to_struct({"refit_grad": (0, 0, 1)}) if form == "stored" else None)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(calls):
        e0.record(stream)
        ctx.tpc_refit_grad(cl, tr, th, s_chi2, grad, w, anchor, 1)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    st = ctx.tpc_sync_status()
    ctx.close()
    assert st == 0, st
    return {"adjoint_form": form, "tracks": nt, "ms_per_call": float(np.median(ts)), "calls": calls,
            "note": "--only-adjoint (profiling run)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the cached launch shapes (or the library defaults) instead of tuning")
    ap.add_argument("--store-tuning", default=None, help="write the autotuned shapes to this JSON cache")
    ap.add_argument("--only-step", action="store_true",
                    help="time the batched step only (no plain/adjoint/e2e/CPU legs); for profiling")
    ap.add_argument("--only-adjoint", default=None, choices=["checkpoints", "stored"],
                    help="time the refit + adjoint of the central calibration event only, in one form; "
                         "for profiling")
    ap.add_argument("--fp32-peak", action="store_true",
                    help="measure the FP32 FMA throughput of the GPU only (the roof of the Kalman stages)")
    args = ap.parse_args()
    if args.fp32_peak:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"fp32_peak": fp32_peak(seconds=2.0)}), flush=True)
        return
    if args.only_adjoint:
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(adjoint_event(args.only_adjoint)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    res = run_native(args, rank, world)
    if rank == 0 and args.only_step:
        pm, pn = res["prof"]
        print(json.dumps({"metric": METRIC, "value": res["n_clusters_all"] / (res["ms_step"] * 1e-3),
                          "unit": "clusters/s", "ms_per_step": res["ms_step"], "steps": args.steps,
                          "stage_ms": {k: v / max(pn, 1) for k, v in pm.items()},
                          "note": "--only-step (profiling run)"}), flush=True)
    elif rank == 0:
        line = finish_native(args, res, world)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(make_batch(args.events, 2000))
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
