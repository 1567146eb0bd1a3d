#!/usr/bin/env python
"""Throughput of GB300 TPC sector track finding (clusters/s).

Default workload: 128 Pb-Pb-like collisions of uneven multiplicity
(b uniform in 0-15 fm, N_tracks = max(10, 9000 (1 - b/15)^2), 36 sectors
each; about 5.5e7 clusters), tracked by the batched form (graph-captured
launch of the whole step chain) in the mixed precision.  A step is one
pass of all tracking steps over the whole batch.  Inputs are resident in
HBM when the timed region starts; they are larger than L2 (~0.8 GB), so no
L2 flush is needed between steps.

Also reported: per-step-boundary times from CUDA events recorded inside the
graph, the roofline of the dominant kernel, the plain per-collision form on
the same batch, end-to-end throughput through host buffers, SM clocks during
the timed region, and the CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle (the only reference there is) on the
host cores.  Multi-GPU: one process per GPU (torchrun); each rank tracks its
own batch (independent collisions, no collective); value = all clusters / the
slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STAGES = ["grid", "neighbours", "clean_start", "tracklets", "selection", "refit"]
# FP64 flops of the mixed-precision tracklet filter: a helix step transports
# the covariance (51 multiply-adds; the float increments go to the
# double-float state on the FP32 pipes); a chi2 test has none (residuals and
# chi2 in float); an update is two scalar updates (the measurement covariance
# is diagonal), each forming S (1), 1/S (1), the gain (5) and the covariance
# (15 multiply-adds)
FLOPS_STEP, FLOPS_TEST, FLOPS_UPDATE = 2 * 51, 0, 2 * (1 + 1 + 5 + 30)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "fp64", "mixed_df"])
    ap.add_argument("--collisions", type=int, default=128)
    ap.add_argument("--workload", default="batch", choices=["batch", "central"],
                    help="batch: the collisions above; central: one central Pb-Pb-like event (small case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-merge", action="store_true")
    ap.add_argument("--no-central", action="store_true", help="skip the central-event sub-record")
    ap.add_argument("--no-clusters", action="store_true")
    ap.add_argument("--no-compression", action="store_true")
    ap.add_argument("--only-clusters", action="store_true",
                    help="time only the cluster-finding leg (central-event digits x4)")
    ap.add_argument("--tuning-cache", default=None, help="autotuner cache file (default: a fresh temp file)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variants", default="mixed_df", help="comma-separated extra precisions timed in the same run")
    ap.add_argument("--frames", type=int, default=30, help="time frames of 16-256 collisions per serving run")
    ap.add_argument("--small-frames", type=int, default=200, help="time frames of 1-8 collisions per serving run")
    ap.add_argument("--serve-loads", default="0.5,0.9,1.1", help="arrival rate / measured capacity, swept")
    ap.add_argument("--only-serving", action="store_true", help="the serving sweep alone (after the capacity step)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)

    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank):
    import synth
    if args.workload == "central":
        return synth.generate_config(1, instance=rank)
    return synth.generate_config(3, instance=rank, n_collisions=args.collisions,
                                 workers=min(16, os.cpu_count() or 1))


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms, clusters, world, device=None):
    """Whole-job numbers of a weak-scaling run: the slowest rank's time per
    step and the clusters of all ranks (every rank tracks its own batch)."""
    if world <= 1:
        return float(ms), int(clusters)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([int(clusters)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def tracklet_traffic(helix_steps):
    """DRAM bytes per launch of k_tracklets<1> from the committed ncu capture,
    scaled by helix steps; None if the kernel's sources changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_tracklets_traffic.json")) as f:
            doc = json.load(f)
        h = hashlib.sha256()
        for src in doc["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != doc["sources_sha256"]:
            return None
        return doc["dram_bytes_per_helix_step"] * helix_steps
    except (OSError, KeyError, ValueError):
        return None


FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz


def alg_bytes(n, hits, n_out, k):
    """Algorithmic DRAM bytes of one pass of the tracking path, the count fixed
    before any tuning: per cluster 12 B of input, 24 B of grid scatter write and
    read, 24 B of links written, read and cleaned, 4 B of start flags; per
    tracklet hit 20 B (y, z read, hit id written, weight atomic, weight read);
    4 B per output cluster id and 200 B per track."""
    return 64.0 * n + 20.0 * hits + 4.0 * n_out + 200.0 * k


def time_batched(trk, dc, out, steps, stream):
    """Mean ms per batched step and mean ms per stage over `steps` graph replays
    (CUDA events recorded inside the graph at the stage boundaries)."""
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
    for row in evs:
        for e in row:
            e.record(stream)
    trk.set_stage_events(evs[0])
    trk.track(dc, out, batched=True)      # capture with event nodes (untimed)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        trk.set_stage_events(evs[k])
        trk.track(dc, out, batched=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    stage_ms = {name: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(steps))
                for i, name in enumerate(STAGES)}
    trk.set_stage_events(None)
    return ms, stage_ms


def instance_views(G, dc):
    """One DeviceClusters view per sector instance (the plain per-sector form)."""
    import torch
    offs = dc.sector_offsets.cpu().numpy()
    views = []
    for i in range(offs.shape[0] - 1):
        a, b = int(offs[i]), int(offs[i + 1])
        so = torch.tensor([0, b - a], dtype=torch.int64, device=dc.y.device)
        views.append(G.DeviceClusters(dc.x[a:b], dc.y[a:b], dc.z[a:b], dc.charge[a:b],
                                      dc.row[a:b] if dc.row is not None else None, so))
    return views


def time_plain(trk, parts, stream, reps):
    """ms of one pass of the plain form: one tpct_track call per part, in turn."""
    import torch
    pout = trk.make_output(max(p.n for p in parts))
    for p in parts[:3]:
        trk.track(p, pout)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        for p in parts:
            trk.track(p, pout)
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / reps


def roofs(ms_step, ms_tracklets, n, gdbg, gout, probe):
    """HBM fraction of the whole step (algorithmic bytes) and FP64 fractions of
    the tracklet stage (algorithmic FP64 flops) against the in-run probe and the
    nominal rate."""
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hits = int(np.asarray(gdbg["tl_nhits"]).sum())
    b = alg_bytes(n, hits, int(gout["n_ids"]), int(gout["n_tracks"]))
    steps, updates, tests = (int(v) for v in gdbg["counters"][:3])
    flops = steps * FLOPS_STEP + tests * FLOPS_TEST + updates * FLOPS_UPDATE
    fp64 = flops / (ms_tracklets * 1e-3) / 1e12
    return {"alg_bytes_per_step": b, "tracklet_hits": hits, "hbm_achieved_gbs": b / (ms_step * 1e-3) / 1e9,
            "hbm_peak_gbs": hbm_peak, "hbm_frac": b / (ms_step * 1e-3) / 1e9 / hbm_peak,
            "hbm_peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "fallback",
            "fp64_flops_tracklets": flops, "fp64_achieved_tflops": fp64,
            "fp64_probe_tflops": probe, "fp64_probe_frac": fp64 / probe if probe else None,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS, "fp64_nominal_frac": fp64 / FP64_NOMINAL_TFLOPS}


def central_leg(args, G, dev, stream, cache, probe):
    """The central Pb-Pb-like event (one collision, 36 sectors, ~1.33 M
    clusters): batched and plain forms, rooflines, and the CUDA result checked
    against the oracle on the whole event."""
    import torch
    import synth
    import oracle
    from oracle.check import compare
    ev = synth.generate_config(1)
    cuts = G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode)
    trk = G.Tracker(precision=args.precision, bz=ev.bz, cuts=cuts, device=dev)
    trk.reserve(ev.n, ev.n_instances)
    dc = G.DeviceClusters.from_event(ev, device=dev)
    out = trk.make_output(ev.n)
    tuning = None if args.no_autotune else trk.autotune(dc, out, cache_path=cache)
    for _ in range(max(3, args.warmup)):
        trk.track(dc, out, batched=True)
    torch.cuda.synchronize()
    status = trk.device_status()
    dbg = trk.debug(ev.n)
    torch.cuda.synchronize()
    gdbg, gout = dbg.to_host(), out.to_host()
    ms, stage_ms = time_batched(trk, dc, out, max(10, args.steps), stream)
    per_sector = time_plain(trk, instance_views(G, dc), stream, 3)
    one_call = time_plain(trk, [dc], stream, 5)
    t0 = time.perf_counter()
    ores = oracle.track_event(ev)
    t_oracle = time.perf_counter() - t0
    rep = compare(ev, ores, gdbg, gout)
    parity = {k: rep[k] for k in ("pass", "nf_mismatch", "nf_excused", "tracklet_mismatch", "tracklet_unexcused",
                                  "tracklets_compared", "track_mismatch", "track_excused", "track_unexcused",
                                  "tracks_oracle", "tracks_gpu", "eff_oracle", "eff_gpu", "param_max_rel_err",
                                  "cov_max_rel_err", "param_plain_rel_err", "cov_diag_plain_rel_err")}
    nt = int(gout["n_tracks"])
    return {"workload": "one central Pb-Pb-like event, 9000 tracks, 36 sectors", "clusters": ev.n,
            "tracks": nt, "precision": args.precision, "tuning": tuning, "device_status": status,
            "batched": {"value": ev.n / (ms * 1e-3), "unit": "clusters/s", "ms_per_event": ms,
                        "tracks_per_s": nt / (ms * 1e-3), "stage_ms": stage_ms},
            "plain_per_sector": {"value": ev.n / (per_sector * 1e-3), "unit": "clusters/s", "ms_per_event": per_sector,
                                 "form": "one tpct_track call per sector instance (36 calls)",
                                 "batched_speedup": per_sector / ms},
            "plain_one_call": {"value": ev.n / (one_call * 1e-3), "unit": "clusters/s", "ms_per_event": one_call,
                               "form": "one tpct_track call for the event (36 instances)",
                               "batched_speedup": one_call / ms},
            "roofline": roofs(ms, stage_ms["tracklets"], ev.n, gdbg, gout, probe),
            "parity_full_event": parity, "oracle_s": t_oracle}


def tracklet_issue(helix_steps, ms, sm_mhz):
    """Issue-slot use of the double-float tracklet kernel: its warp
    instructions (the committed ncu count per helix step, scaled by this run's
    helix steps) over the issue slots of 152 SMs x 4 schedulers in its
    CUDA-event time at the sampled SM clock; None if the kernel's sources
    changed since the count was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_tracklets_df_issue.json")) as f:
            doc = json.load(f)
        h = hashlib.sha256()
        for src in doc["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != doc["sources_sha256"]:
            return None
    except (OSError, KeyError, ValueError):
        return None
    mhz = sm_mhz or 2070.0
    instr = doc["warp_instructions_per_helix_step"] * helix_steps
    slots = 152 * 4 * ms * 1e-3 * mhz * 1e6
    return {"warp_instructions": instr, "issue_slots": slots, "issue_frac": instr / slots,
            "sm_mhz": mhz, "source": "profiles/k_tracklets_df_issue.json"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(ev, gpu_out, gpu_dbg, budget_s=20.0):
    """Oracle on a bounded sample of the workload's sector instances (rank 0,
    N = 1); also checks the CUDA result on the same sample."""
    import oracle
    from oracle.check import compare
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_util import slice_instances
    rng = np.random.default_rng(12345)
    order = rng.permutation(ev.n_instances)
    sizes = np.diff(ev.sector_offsets)
    # about budget_s of single-thread work at ~2.5e5 clusters/s
    target = int(budget_s * 2.5e5)
    take, tot = [], 0
    for i in order:
        take.append(int(i))
        tot += int(sizes[i])
        if tot >= target:
            break
    idx = np.sort(np.array(take))
    sub = ev.select_instances(idx)
    t0 = time.perf_counter()
    ores = oracle.track_event(sub)
    dt = time.perf_counter() - t0
    rep = None
    if gpu_out is not None:
        tr, dbg = slice_instances(ev, gpu_out, gpu_dbg, idx)
        r = compare(sub, ores, dbg, tr)
        rep = {k: r[k] for k in ("pass", "nf_mismatch", "nf_excused", "tracklet_mismatch", "tracklet_unexcused",
                                 "tracklets_compared", "track_mismatch", "track_excused", "track_unexcused",
                                 "tracks_oracle", "tracks_gpu", "eff_oracle", "eff_gpu", "cov_max_rel_err",
                                 "param_plain_rel_err", "cov_diag_plain_rel_err")}
        rep["param_max_rel_err"] = max(r["param_max_rel_err"])
    return {"value": sub.n / dt, "unit": "clusters/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(idx)} of {ev.n_instances} sector instances ({sub.n} clusters), "
                      f"single-threaded FP64, {dt:.1f} s"}, rep, idx


def merge_leg(args, ev, G, trk, dc, out, stream):
    """Cross-sector merging of the tracked batch: mean CUDA-event time of
    tpct_merge over a few calls on the resident tracks."""
    import torch
    sec = np.asarray(ev.sectors, dtype=np.int32)
    evi = (np.arange(ev.n_instances) // ev.sectors_per_event).astype(np.int32)
    n_events = int(evi.max()) + 1
    ch = trk.merge(dc, out, sec, evi, n_events)
    for _ in range(2):
        trk.merge(dc, out, sec, evi, n_events, out=ch)
    torch.cuda.synchronize()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    m0.record(stream)
    for _ in range(reps):
        trk.merge(dc, out, sec, evi, n_events, out=ch)
    m1.record(stream)
    torch.cuda.synchronize()
    mms = m0.elapsed_time(m1) / reps
    n_tracks = int(out.counts[0].item())
    n_chains = int(ch.counts[0].item())
    return {"ms": mms, "tracks_in": n_tracks, "chains": n_chains,
            "tracks_per_s": n_tracks / (mms * 1e-3), "device_status": trk.device_status()}


def compression_leg(args, ev, G, trk, dc, out, stream, reps=5):
    """Track-model compression of the batch's clusters with its tracks, and
    the GPU decoding of the stream: size per cluster, mean CUDA-event times,
    and the decoder's HBM roofline (algorithmic bytes: the stream read, 15 B
    written per cluster)."""
    import torch
    st = trk.tm_encode(dc, out)
    torch.cuda.synchronize()
    nt = int(out.counts[0].item())
    nb = int(st["n_bytes"].item())
    cap = st["data"].numel()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        trk.tm_encode(dc, out, capacity_bytes=cap)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        trk.tm_encode(dc, out, capacity_bytes=cap)
    e1.record(stream)
    torch.cuda.synchronize()
    enc_ms = e0.elapsed_time(e1) / reps
    d = trk.tm_decode(st["data"], st["track_offsets"], nt, st["row_offsets"], ev.n_instances, ev.n)
    for _ in range(2):
        trk.tm_decode(st["data"], st["track_offsets"], nt, st["row_offsets"], ev.n_instances, ev.n)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        trk.tm_decode(st["data"], st["track_offsets"], nt, st["row_offsets"], ev.n_instances, ev.n)
    e1.record(stream)
    torch.cuda.synchronize()
    dec_ms = e0.elapsed_time(e1) / reps
    ok = int(d["n"].item()) == ev.n
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    dec_bytes = nb + 15.0 * ev.n
    return {"clusters": ev.n, "tracks": nt, "bytes": nb, "bytes_per_cluster": nb / ev.n,
            "raw_bytes_per_cluster": 15, "encode_ms": enc_ms, "decode_ms": dec_ms,
            "encode_clusters_per_s": ev.n / (enc_ms * 1e-3), "decode_clusters_per_s": ev.n / (dec_ms * 1e-3),
            "decoded_all": ok,
            "decode_roofline": {"bound": "hbm", "kernel": "k_td_decode", "achieved": dec_bytes / (dec_ms * 1e-3) / 1e9,
                                "peak": peak, "unit": "GB/s", "frac": dec_bytes / (dec_ms * 1e-3) / 1e9 / peak}}


def cluster_leg(args, G, dev, stream, copies=4, reps=10):
    """Cluster finding (the step upstream of track finding) on the digits of
    the central Pb-Pb-like event, replicated `copies` times as independent
    collisions so that the input (~430 MB) exceeds L2; mean CUDA-event time of
    tpct_find_clusters over `reps` calls after 3 warm-ups."""
    import torch
    import synth.digits as D
    dg = D.generate_digits(1, workers=min(16, os.cpu_count() or 1))
    n_rk = dg.row_offsets.shape[0] - 1
    offs = np.concatenate([dg.row_offsets[:-1] + c * dg.n for c in range(copies)] + [[copies * dg.n]])
    rep = D.Digits(pad=np.tile(dg.pad, copies), time=np.tile(dg.time, copies), adc=np.tile(dg.adc, copies),
                   row_offsets=offs.astype(np.int64), sectors=np.tile(dg.sectors, copies), readout=dg.readout,
                   n_pad=dg.n_pad, truth={})
    trk = G.Tracker(precision="mixed", device=dev)
    dd = G.DeviceDigits.from_digits(rep, device=dev)
    out = trk.find_clusters(dd)
    for _ in range(2):
        trk.find_clusters(dd, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        trk.find_clusters(dd, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    h = out.counts.cpu().numpy()
    n_cl = int(h[0])
    # algorithmic bytes: pad, time, adc (6 B) per digit, one row offset (8 B)
    # per row, the 36 B of each cluster written
    bytes_alg = 6.0 * rep.n + 8.0 * (copies * n_rk + 1) + 36.0 * n_cl
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    ach = bytes_alg / (ms * 1e-3) / 1e9
    return {"workload": f"central Pb-Pb-like event digits x{copies} ({rep.n} digits, {copies * n_rk} pad rows)",
            "ms": ms, "digits_per_s": rep.n / (ms * 1e-3), "clusters": n_cl, "clusters_per_s": n_cl / (ms * 1e-3),
            "status": int(h[1]),
            "roofline": {"bound": "hbm", "kernel": "k_clusterer", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes_per_launch": bytes_alg}}


def make_frames(pool, n_frames, k_range, rng, pin):
    """Frames of k collisions, k uniform in k_range, each a random run of
    consecutive collisions of the pool (pinned host views)."""
    ne, spe, offs = pool.n_events, pool.sectors_per_event, pool.sector_offsets
    import torch
    frames = []
    for _ in range(n_frames):
        k = int(rng.integers(k_range[0], min(k_range[1], ne) + 1))
        c0 = int(rng.integers(0, ne - k + 1))
        a, b = int(offs[c0 * spe]), int(offs[(c0 + k) * spe])
        so = torch.from_numpy((offs[c0 * spe:(c0 + k) * spe + 1] - a).astype(np.int64)).pin_memory()
        frames.append(dict(x=pin["x"][a:b], y=pin["y"][a:b], z=pin["z"][a:b], charge=pin["charge"][a:b],
                           row=pin["row"][a:b], sector_offsets=so, collisions=k))
    return frames


def serve_run(G, args, cuts, bz, frames, rate, slots, seed):
    """Frames arriving as a Poisson process of `rate` Hz into the serving
    runtime with `slots` slots; a consumer thread releases every frame once it
    is done (in submission order), so only frames in flight hold the arena.
    Latency = submission -> results ready, as seen by the runtime."""
    import threading
    sizes = np.array([f["y"].shape[0] for f in frames], np.float64)
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, len(frames))
    arrive = np.cumsum(gaps) - gaps[0]
    srv = G.Server(n_slots=slots, budget_bytes=int(args.serve_budget_gb * (1 << 30)), precision=args.precision,
                   bz=bz, cuts=cuts)
    for f in frames[:2]:                      # warm-up
        tk = srv.submit(f)
        srv.wait(tk)
        srv.release(tk)
    tks = []
    lat = np.zeros(len(frames))
    done = np.zeros(len(frames))
    status = []

    def consumer():
        for i in range(len(frames)):
            while len(tks) <= i:
                time.sleep(0.0005)
            srv.wait(tks[i])
            info = srv.poll(tks[i])
            lat[i] = info["latency_us"] / 1e3
            done[i] = time.perf_counter()
            status.append(info["status"])
            srv.release(tks[i])

    th = threading.Thread(target=consumer)
    th.start()
    t0 = time.perf_counter()
    for f, ta in zip(frames, arrive):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tks.append(srv.submit(f))
    th.join()
    end = done.max() - t0
    st = srv.stats()
    srv.close()
    del srv
    return {"slots": slots, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "sustained_clusters_per_s": float(sizes.sum() / end), "offered_clusters_per_s": float(sizes.sum() / arrive[-1])
            if arrive[-1] > 0 else None, "peak_in_flight": st["peak_in_flight"], "peak_gb": st["peak_bytes"] / 2 ** 30,
            "retries": st["retries"], "failed": int(sum(1 for x in status if x != 0))}


def serving_leg(args, pool, G, capacity_cps):
    """Serving of time frames of 16-256 collisions drawn from a 256-collision
    pool (the batching generator), arriving as a Poisson process, at several
    loads (arrival rate x mean frame size / the measured batched capacity),
    with one slot (frames one after another: the plain per-frame form) and
    three slots (continuous batching); plus a mix of small frames (1-8
    collisions), where one frame does not fill the GPU."""
    import torch
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(pool, k))).pin_memory()
           for k in ("x", "y", "z", "charge", "row")}
    cuts = G.default_cuts(sig_readout=pool.sigma.at_readout, sig_cathode=pool.sigma.at_cathode)
    loads = [float(v) for v in args.serve_loads.split(",") if v]
    out = {"budget_gb": args.serve_budget_gb, "pool_collisions": pool.n_events, "capacity_clusters_per_s": capacity_cps}
    for name, n_frames, k_range, seed in (("frames_16_256", args.frames, (16, 256), 4000),
                                          ("frames_1_8", args.small_frames, (1, 8), 4100)):
        if n_frames <= 0:
            continue
        frames = make_frames(pool, n_frames, k_range, np.random.default_rng(seed), pin)
        sizes = np.array([f["y"].shape[0] for f in frames], np.float64)
        coll = [f["collisions"] for f in frames]
        rec = {"frames": len(frames), "collisions_per_frame": [int(min(coll)), int(max(coll))],
               "mean_frame_clusters": float(sizes.mean()), "max_frame_clusters": float(sizes.max()), "sweep": []}
        for load in (loads if name == "frames_16_256" else [0.9]):
            rate = load * capacity_cps / sizes.mean()
            for slots in (1, 3):
                r = serve_run(G, args, cuts, pool.bz, frames, rate, slots, seed + int(load * 100))
                r.update(load=load, arrival_rate_hz=rate)
                rec["sweep"].append(r)
        out[name] = rec
    return out


def publishing_leg(args, ev, G, capacity_cps, n_frames=48):
    """An offline source publishing frames of 8-32 collisions cut from the
    batch into the serving runtime (3 slots), followed by a serial host
    consumer that fetches every frame's tracks and spends 1.25x the frame's
    GPU time on it (the slower serial stage of Section 3), driven by the
    native pacer with the naive policy (in-flight limit only) and with
    publishing-rate smoothing.  Latency = publication -> consumed."""
    import torch
    ne, spe, offs = ev.n_events, ev.sectors_per_event, ev.sector_offsets
    rng = np.random.default_rng(5000)
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(ev, k))).pin_memory()
           for k in ("x", "y", "z", "charge", "row")}
    frames = []
    for _ in range(n_frames):
        k = int(rng.integers(8, min(32, ne) + 1))
        c0 = int(rng.integers(0, ne - k + 1))
        a, b = int(offs[c0 * spe]), int(offs[(c0 + k) * spe])
        so = torch.from_numpy((offs[c0 * spe:(c0 + k) * spe + 1] - a).astype(np.int64)).pin_memory()
        frames.append(dict(x=pin["x"][a:b], y=pin["y"][a:b], z=pin["z"][a:b], charge=pin["charge"][a:b],
                           row=pin["row"][a:b], sector_offsets=so))
    sizes = np.array([f["y"].shape[0] for f in frames], np.float64)
    cost = 1.25 * sizes / capacity_cps
    cuts = G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode)
    limit = 12
    out = {"frames": n_frames, "mean_frame_clusters": float(sizes.mean()), "max_in_flight": limit,
           "consumer_s_per_frame": float(cost.mean())}
    for policy in ("naive", "smooth"):
        srv = G.Server(n_slots=3, budget_bytes=int(args.serve_budget_gb * (1 << 30)), precision=args.precision,
                       bz=ev.bz, cuts=cuts)
        for f in frames[:2]:                      # warm-up
            srv.wait(srv.submit(f))
        for tk in list(srv._frames):
            srv.release(tk)
        pacer = G.Pacer(policy, max_in_flight=limit, initial_delay_s=float(cost.mean()) * 0.25)
        lock = threading.Lock()
        tks, t_pub, t_done = [], [], [0.0] * n_frames
        state = {"consumed": 0}
        done0 = srv.stats()["completed"]

        def backlog():
            st = srv.stats()
            waiting = (st["completed"] - done0) - state["consumed"]
            return st["queued"] + max(0, waiting - 2)

        def consumer():
            for i in range(n_frames):
                while True:
                    with lock:
                        if len(tks) > i:
                            tk = tks[i]
                            break
                    time.sleep(0.0005)
                srv.wait(tk)
                srv.fetch(tk)
                time.sleep(cost[i])
                srv.release(tk)
                now = time.perf_counter()
                with lock:
                    t_done[i] = now
                    state["consumed"] += 1
                    pacer.on_consumed(now, len(tks) - state["consumed"], backlog())

        th = threading.Thread(target=consumer)
        t0 = time.perf_counter()
        th.start()
        samples = []
        while len(tks) < n_frames:
            now = time.perf_counter()
            with lock:
                inflight = len(tks) - state["consumed"]
                ok, wait = pacer.try_publish(now, inflight, backlog())
                if ok:
                    tks.append(srv.submit(frames[len(tks)]))
                    t_pub.append(now)
            samples.append(inflight)
            if not ok:
                time.sleep(min(wait, 0.002) if wait > 0 else 0.001)
        while th.is_alive():
            with lock:
                samples.append(len(tks) - state["consumed"])
            time.sleep(0.001)
        th.join()
        t_end = max(t_done)
        lat = (np.array(t_done) - np.array(t_pub)) * 1e3
        st = srv.stats()
        out[policy] = {"makespan_s": t_end - t0, "clusters_per_s": float(sizes.sum() / (t_end - t0)),
                       "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                       "mean_in_flight": float(np.mean(samples)), "peak_gb": st["peak_bytes"] / 2 ** 30,
                       "final_delay_s": pacer.delay, "pressure_events": pacer.pressure_events}
        srv.close()
        del srv
    return out


def _oracle_chunk(payload):
    import oracle
    import synth
    y, z, row, offs, sig = payload
    ev = synth.Event(x=None, y=y, z=z, charge=None, row=row, sector_offsets=offs, sectors=None, mc=None,
                     sigma=synth.events.SigmaModel(*sig))
    t0 = time.perf_counter()
    oracle.track_event(ev)
    return time.perf_counter() - t0


def cpu_baseline_parallel(ev, idx, workers):
    """The same oracle, unchanged, over the same sample split into independent
    sector instances, on a spawn process pool of all host cores."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunks = np.array_split(np.asarray(idx), workers * 4)
    payloads = []
    for ch in chunks:
        if len(ch) == 0:
            continue
        sub = ev.select_instances(ch)
        payloads.append((sub.y, sub.z, sub.row, sub.sector_offsets,
                         (ev.sigma.at_readout, ev.sigma.at_cathode, ev.sigma.z_max)))
    n = sum(int(p[3][-1]) for p in payloads)
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_chunk, payloads[:workers]))          # start-up and warm-up
        t0 = time.perf_counter()
        list(ex.map(_oracle_chunk, payloads))
        dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "clusters/s", "cores": workers, "kind": "oracle",
            "sample": f"the same {len(idx)} sector instances ({n} clusters) on {workers} processes, {dt:.1f} s"}


METRIC = "TPC clusters/s tracked (batched, mixed FP32/FP64)"


def workload_name(args):
    return (f"{args.collisions} collisions, b uniform 0-15 fm, 36 sectors each"
            if args.workload == "batch" else "one central Pb-Pb-like event, 9000 tracks")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    # a bounded sample of the same workload: the first collisions of the batch
    ncoll = max(1, min(args.collisions, 4))
    ev = synth.generate_config(3, instance=0, n_collisions=ncoll)
    per_step = []
    for s in range(args.warmup + args.steps):
        k = s % ev.n_instances
        idx = np.arange(k, min(ev.n_instances, k + 36))
        sub = ev.select_instances(idx)
        t0 = time.perf_counter()
        oracle.track_event(sub)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per_step.append((sub.n, dt))
    n = sum(a for a, _ in per_step)
    t = sum(b for _, b in per_step)
    v = n / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "clusters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "precision": "fp64 (the oracle)",
                       "form": "single-threaded CPU oracle, a bounded sample of 36 sector instances per step"},
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(per_step)} steps of 36 sector instances ({n} clusters)"},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    if args.only_clusters:
        # the cluster-finding leg alone (profiling aid): one JSON object
        import torch
        import paper_2502_09138_gb300 as G
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        leg = cluster_leg(args, G, dev, torch.cuda.current_stream(dev), reps=max(1, args.steps))
        if rank == 0:
            print(json.dumps({"cluster_finding": leg}), flush=True)
        return
    # generate before any CUDA call (the generator uses a spawn process pool)
    ev = workload(args, rank)
    pool = None
    if not args.no_serving and args.workload == "batch":
        # the serving frames (16-256 collisions) come from a pool of 256
        # collisions: the batch plus further collisions of the same generator
        import synth
        extra = 256 - ev.n_events
        pool = ev if extra <= 0 else synth.concat_events([ev, synth.generate_config(
            3, instance=rank + 1000, n_collisions=extra, workers=min(16, os.cpu_count() or 1))])
    import torch
    import paper_2502_09138_gb300 as G
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cuts = G.default_cuts(sig_readout=ev.sigma.at_readout, sig_cathode=ev.sigma.at_cathode)
    trk = G.Tracker(precision=args.precision, bz=ev.bz, cuts=cuts, device=dev)
    trk.reserve(ev.n, ev.n_instances)
    dc = G.DeviceClusters.from_event(ev, device=dev)
    out = trk.make_output(ev.n, cap_tracks=ev.n // 20 + 1024, cap_ids=ev.n)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    tuning = None
    import tempfile
    cache = args.tuning_cache or os.path.join(tempfile.gettempdir(), f"tpct_tuning_{os.getpid()}.cache")
    if not args.no_autotune:
        tuning = trk.autotune(dc, out, cache_path=cache)
    # warm-up (also builds the graph)
    for _ in range(args.warmup):
        trk.track(dc, out, batched=True)
    torch.cuda.synchronize()
    st = trk.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")
    dbg = trk.debug(ev.n)
    torch.cuda.synchronize()
    gdbg = dbg.to_host()
    gout = out.to_host()

    launches0 = trk.kernel_launches()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ms, stage_ms = time_batched(trk, dc, out, args.steps, stream)
    barrier()
    clocks = sampler.stop()
    # the capture replay inside time_batched launches one untimed step
    launches = (trk.kernel_launches() - launches0) * args.steps // (args.steps + 1)
    ms, n_total = aggregate_ranks(ms, ev.n, world, dev)
    value = n_total / (ms * 1e-3)
    n_tracks = int(gout["n_tracks"])
    if args.only_serving:
        # the serving sweep alone, against the capacity just measured
        if rank == 0:
            print(json.dumps({"capacity_clusters_per_s": value / world, "ms_per_step": ms,
                              "serving": serving_leg(args, pool, G, value / world)}), flush=True)
        return

    # roofline of the dominant kernel
    peaks = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    steps, updates, tests = (int(v) for v in gdbg["counters"][:3])
    fp64_flops = steps * FLOPS_STEP + tests * FLOPS_TEST + updates * FLOPS_UPDATE
    blocks = 152 * 16
    pm = G.probe_fma(True, blocks, 2048)
    fp64_probe = 2.0 * 8 * 2048 * blocks * 256 / (pm * 1e-3) / 1e12
    step_roofs = roofs(ms, stage_ms["tracklets"], ev.n, gdbg, gout, fp64_probe)
    roofline = None
    if dom == "tracklets" and args.precision == "mixed":
        # FP64-bound: the peak is the unit-count rate at the SM clock sampled
        # during the timed steps (152 SMs x 2 FP64 FMA per clock x 2 flops);
        # the in-run FMA probe, whose chains reach ~85 % of it, is context
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        fp64_peak = 152 * 2 * 2 * mhz * 1e6 / 1e12
        ach = fp64_flops / (stage_ms["tracklets"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_tracklets (FP64 covariance arithmetic)", "achieved": ach,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                    "traffic": tracklet_traffic(steps) if args.precision == "mixed" else None,
                    "peak_source": f"FP64 unit count x sampled SM clock (152 SMs x 2 FMA/clk x 2 flops x {mhz:.0f} MHz)",
                    "algorithmic_flops_per_launch": fp64_flops,
                    "fp64_probe_tflops": fp64_probe, "fp64_probe_frac": ach / fp64_probe,
                    "fp64_nominal_frac": ach / FP64_NOMINAL_TFLOPS,
                    "hbm_frac": step_roofs["hbm_frac"], "hbm_achieved_gbs": step_roofs["hbm_achieved_gbs"],
                    "hbm_peak_gbs": step_roofs["hbm_peak_gbs"],
                    "hbm_alg_bytes_per_step": step_roofs["alg_bytes_per_step"]}
    else:
        bytes_alg = step_roofs["alg_bytes_per_step"]
        ach = bytes_alg / (stage_ms[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peaks.get("hbm_gbs", 6800.0),
                    "unit": "GB/s", "frac": ach / peaks.get("hbm_gbs", 6800.0), "traffic": None,
                    "hbm_frac": step_roofs["hbm_frac"], "fp64_nominal_frac": step_roofs["fp64_nominal_frac"]}

    line = {
        "metric": METRIC, "value": value, "unit": "clusters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # arithmetic types of the path: float transport and search; FP64
        # tracklet covariance update and refit head; double-float (float pairs)
        # tracklet state and refit passes, and the tracklet covariance in mixed_df
        "dtype": {"mixed": "f32+f64+df64", "fp32": "f32", "fp64": "f64", "mixed_df": "f32+df64+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "clusters_per_rank": ev.n, "sector_instances": ev.n_instances, "precision": args.precision,
                   "form": "batched (graph-captured step chain)", "l2": "inputs 0.8 GB > L2, no flush",
                   "parallelism": f"replicas x{world} (independent collisions)"},
        "tracks_per_s": n_tracks * world / (ms * 1e-3), "tracks": n_tracks, "tuning": tuning,
        "stage_ms": stage_ms, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
        "counters": {"helix_steps": steps, "kalman_updates": updates, "chi2_tests": tests},
    }

    # plain per-collision form on the same batch
    if not args.no_plain:
        offs = ev.sector_offsets
        spe = ev.sectors_per_event
        parts = []
        for c in range(ev.n_events):
            a, b = int(offs[c * spe]), int(offs[(c + 1) * spe])
            so = torch.from_numpy((offs[c * spe:(c + 1) * spe + 1] - a).astype(np.int64)).to(dev)
            parts.append(G.DeviceClusters(dc.x[a:b], dc.y[a:b], dc.z[a:b], dc.charge[a:b], dc.row[a:b], so))
        pms = time_plain(trk, parts, stream, max(1, min(3, args.steps)))
        sms = time_plain(trk, instance_views(G, dc), stream, 2)
        line["plain"] = {"value": ev.n / (pms * 1e-3), "ms_per_step": pms, "unit": "clusters/s",
                         "form": "one tpct_track call per collision (36 instances), plain launches",
                         "batched_speedup": pms / ms,
                         "per_sector": {"value": ev.n / (sms * 1e-3), "ms_per_step": sms, "unit": "clusters/s",
                                        "form": f"one tpct_track call per sector instance ({ev.n_instances} calls)",
                                        "batched_speedup": sms / ms}}

    # end to end through host buffers
    if not args.no_e2e:
        # the inputs the tracking step reads: y, z, row and the instance
        # offsets (x is read only without the row; charge not at all)
        in_keys = ("y", "z", "row", "sector_offsets")
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(ev, k))).pin_memory() for k in ("y", "z", "row")}
        host["sector_offsets"] = torch.from_numpy(ev.sector_offsets.astype(np.int64)).pin_memory()
        dce = G.DeviceClusters.from_event(ev, device=dev, tracking_only=True)
        res_host = {k: torch.empty(getattr(out, k).shape, dtype=getattr(out, k).dtype).pin_memory()
                    for k in ("counts", "n_cl", "offset", "param", "cov", "chi2", "cluster_ids")}
        d2h = sum(int(t.numel() * t.element_size()) for k, t in res_host.items())
        h2d = sum(int(t.numel() * t.element_size()) for t in host.values())
        def e2e_step():
            for k in in_keys:
                getattr(dce, k).copy_(host[k], non_blocking=True)
            trk.track(dce, out, batched=True)
            for k, t in res_host.items():
                t.copy_(getattr(out, k), non_blocking=True)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, min(5, args.steps))
        b0.record(stream)
        for _ in range(reps):
            e2e_step()
        b1.record(stream)
        torch.cuda.synchronize()
        ems = b0.elapsed_time(b1) / reps
        serial = {"value": ev.n * world / (ems * 1e-3), "unit": "clusters/s", "ms_per_step": ems,
                  "form": "one stream: copy in, track, copy out"}
        # Pipelined: two trackers (own workspace, inputs, outputs, stream)
        # take the steps in turn, so one step's host copies overlap the other
        # step's kernels; every step still copies its inputs in and its result
        # out inside the timed region.  A step's result is its track count
        # and id count (copied with the step) and then the filled rows of its
        # outputs: the host reads a lane's counts only after it has queued the
        # next lane's step, so the GPU never waits for the host.
        trk2 = G.Tracker(precision=args.precision, bz=ev.bz, cuts=cuts, device=dev)
        trk2.reserve(ev.n, ev.n_instances)
        if tuning:
            trk2.set_tuning(tuning["clusters_per_bin"], tuning["tracklet_block"], tuning["refit_block"])
        dc2 = G.DeviceClusters.from_event(ev, device=dev, tracking_only=True)
        out2 = trk2.make_output(ev.n, cap_tracks=ev.n // 20 + 1024, cap_ids=ev.n)
        res_host2 = {k: torch.empty_like(t).pin_memory() for k, t in res_host.items()}
        lanes = [(trk, dce, out, res_host, torch.cuda.Stream(dev)), (trk2, dc2, out2, res_host2, torch.cuda.Stream(dev))]
        row_keys = ("n_cl", "offset", "param", "cov", "chi2")
        copied = [0, 0]

        def e2e_launch(i):
            t_, d_, o_, rh_, s_ = lanes[i % 2]
            with torch.cuda.stream(s_):
                for k in in_keys:
                    getattr(d_, k).copy_(host[k], non_blocking=True)
                t_.track(d_, o_, batched=True, stream=s_)
                rh_["counts"].copy_(o_.counts, non_blocking=True)
                ev_ = torch.cuda.Event()
                ev_.record(s_)
            return ev_

        def e2e_fetch(i, ev_):
            t_, d_, o_, rh_, s_ = lanes[i % 2]
            ev_.synchronize()
            nt = min(int(rh_["counts"][0]), o_.capacity_tracks)
            ni = min(int(rh_["counts"][1]), o_.capacity_ids)
            with torch.cuda.stream(s_):
                for k in row_keys:
                    rh_[k][:nt].copy_(getattr(o_, k)[:nt], non_blocking=True)
                rh_["cluster_ids"][:ni].copy_(o_.cluster_ids[:ni], non_blocking=True)
            copied[0] = int(rh_["counts"].numel() * rh_["counts"].element_size())
            copied[1] = sum(int(rh_[k][:nt].numel() * rh_[k].element_size()) for k in row_keys) + ni * 4

        def e2e_run(n_steps):
            pending = None
            for i in range(n_steps):
                ev_ = e2e_launch(i)
                if pending is not None:
                    e2e_fetch(*pending)
                pending = (i, ev_)
            e2e_fetch(*pending)

        e2e_run(4)
        torch.cuda.synchronize()
        reps_p = 2 * max(2, min(10, args.steps))   # 2x as many as the timed steps: fill and drain amortised
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _, _, _, _, s_ in lanes:
            s_.wait_event(c0)
        e2e_run(reps_p)
        for _, _, _, _, s_ in lanes:
            stream.wait_stream(s_)
        c1.record(stream)
        torch.cuda.synchronize()
        pms_ = c0.elapsed_time(c1) / reps_p
        st2 = trk2.device_status()
        nt_, ni_ = (int(v) for v in res_host["counts"])
        same = (torch.equal(res_host["counts"], res_host2["counts"])
                and torch.equal(res_host["n_cl"][:nt_], res_host2["n_cl"][:nt_])
                and torch.equal(res_host["cluster_ids"][:ni_], res_host2["cluster_ids"][:ni_]))
        line["e2e"] = {"value": ev.n * world / (pms_ * 1e-3), "unit": "clusters/s", "ms_per_step": pms_,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": copied[0] + copied[1],
                       "form": "two trackers on two streams take the steps in turn (copies overlap kernels); "
                               "inputs copied in: y, z, row, instance offsets (what tracking reads); "
                               "the result read back is the counts and the filled output rows",
                       "device_status": st2, "lanes_agree": bool(same),
                       "serial": dict(serial, d2h_bytes_per_step=d2h,
                                      form="one stream: copy in (y, z, row, offsets), track, copy out (whole output buffers)")}
        del trk2, dc2, dce, out2, res_host2, lanes
        torch.cuda.empty_cache()

    # cross-sector merging of the batch's sector tracks (a step after the
    # tracking chain, timed on its own; not part of `value`)
    if not args.no_merge and ev.sectors_per_event > 1:
        line["merge"] = merge_leg(args, ev, G, trk, dc, out, stream)
    if not args.no_clusters:
        line["cluster_finding"] = cluster_leg(args, G, dev, stream)
    if not args.no_compression:
        line["compression"] = compression_leg(args, ev, G, trk, dc, out, stream)

    if not args.no_central and args.workload == "batch":
        line["central"] = central_leg(args, G, dev, stream, cache, fp64_probe)

    variants = {}
    for vp in [v for v in args.variants.split(",") if v and v != args.precision]:
        vt = G.Tracker(precision=vp, bz=ev.bz, cuts=cuts, device=dev)
        vt.reserve(ev.n, ev.n_instances)
        vtun = None if args.no_autotune else vt.autotune(dc, out, cache_path=cache)
        for _ in range(args.warmup):
            vt.track(dc, out, batched=True)
        torch.cuda.synchronize()
        vev = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
        for row_ in vev:
            for e in row_:
                e.record(stream)
        vt.set_stage_events(vev[0])
        vt.track(dc, out, batched=True)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for k in range(args.steps):
            vt.set_stage_events(vev[k])
            vt.track(dc, out, batched=True)
        c1.record(stream)
        torch.cuda.synchronize()
        vms = c0.elapsed_time(c1) / args.steps
        st_v = vt.device_status()
        variants[vp] = {"value": ev.n / (vms * 1e-3), "unit": "clusters/s", "ms_per_step": vms,
                        "device_status": st_v, "tuning": vtun,
                        "stage_ms": {name: statistics.mean(vev[k][i].elapsed_time(vev[k][i + 1])
                                                           for k in range(args.steps))
                                     for i, name in enumerate(STAGES)}}
        if vp == "mixed_df":
            variants[vp]["tracklet_issue"] = tracklet_issue(steps, variants[vp]["stage_ms"]["tracklets"],
                                                            clocks.get("sm_mhz") if clocks else None)
        vt.set_stage_events(None)
        del vt
    if variants:
        line["variants"] = variants

    if not args.no_serving and args.workload == "batch":
        line["serving"] = serving_leg(args, pool, G, value / world)
        line["publishing"] = publishing_leg(args, ev, G, value / world)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, par, idx = cpu_baseline(ev, gout, gdbg)
        line["cpu_baseline"] = cb
        line["parity_on_sample"] = par
        line["cpu_baseline_parallel"] = cpu_baseline_parallel(ev, idx, os.cpu_count() or 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
