#!/usr/bin/env python
"""Throughput benchmark of the GB300 SGM stereo library in MDE/s (Eq. mdes: W * H * D / time).

Default (N = 1): the 1242x375 pair, D = 128, census 9x7, 8 paths, P1 = 10, P2 = 120, LR check and
3x3 median, one res2tac_compute per step on device-resident inputs, L2 flushed between steps
(a 256 MB write outside the per-step events). Also measured in the same run and reported in the
same JSON line:
  - e2e: four pairs of the workload in turn through res2tac_compute_host from pinned host
    buffers (transfers, compute, synchronise; L2 flushed before each step), as the paper times
    its pipeline, and the same with one staged cudaMemcpyAsync per image and for the map;
  - batched: 64 pairs of uneven W, H, D in one res2tac_compute_batch call (persistent kernels
    under a CUDA graph) vs the same 64 pairs as per-pair res2tac_compute launches;
  - serving: 10,000 Poisson arrivals (the batch sizes plus 5 % 3840x2160, D = 256) at each of
    200, 500, 1000, 2000 and 5000 pairs/s through the continuous-batching server, p50 / p99 /
    p99.9 latency per rate; a 1 % sample checked against the CPU oracle after the sweep;
  - roofline of the dominant kernel (path aggregation) from CUDA events recorded around it on its
    own stream, against the measured packed-u16 integer rate (and the measured HBM copy rate);
  - cpu_baseline: the single-threaded C oracle on the same pair, on the host cores.
Under torchrun (N > 1) every rank runs an independent replica (the path does not shard; no
collective touches the data path) and rank 0 prints the aggregate.

--impl reference times the CPU oracle (the only reference implementation: the paper ships no
code) on a bounded band of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "1242x375_d128_ct9x7_r8"
METRIC = "MDE/s (W*H*D*fps/1e6), plain single-pair launches"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch-pairs", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", default="200,500,1000,2000,5000")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--pair", type=int, nargs=3, metavar=("W", "H", "D"), default=None,
                    help="time a seeded road-like pair of this size instead of the 1242x375 "
                         "workload (9x7, 8 paths, LR + median; for profiling larger pairs)")
    ap.add_argument("--profile-steps", type=int, default=0, metavar="N",
                    help="only run N plain steps of the workload and exit, printing nothing "
                         "(the command that ncu captures kernels of)")
    ap.add_argument("--cost-mode", type=int, default=0, choices=[0, 1, 2],
                    help="with --profile-steps: the tuning's cost_mode (0 = default)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="with --profile-steps: each step is res2tac_compute_batch of the pair "
                         "alone, followed by the same pair through res2tac_compute")
    return ap.parse_args()


def _workload_pair(args, seed):
    """(left, right, params, name) of the timed workload: the 1242x375 D=128 pair, or with
    --pair a seeded road-like scene of the given size with the same method settings."""
    from paper_2106_07927_gb300 import scenes
    if args.pair is None:
        left, right, _, prm = scenes.single_pair(WORKLOAD, seed)
        return left, right, prm, WORKLOAD
    W, H, D = args.pair
    left, right, _ = scenes.make_scene("road", 3 + seed, W, H, D)
    return (left, right, scenes.params(W, H, D, 9, 7, 10, 120, 8,
                                        scenes.FLAG_LR_CHECK | scenes.FLAG_MEDIAN),
            f"{W}x{H}_d{D}_ct9x7_r8")


def _traffic(tuning):
    """DRAM bytes (read + write) per launch of the aggregation stage, from the ncu capture recorded
    in profiles/aggregate_traffic.json; None when that capture is missing or was taken with other
    kernel settings than `tuning` (the timed context's res2tac_tuning)."""
    p = os.path.join(ROOT, "profiles", "aggregate_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    want = rec.get("tuning", {})
    if not want or any(getattr(tuning, k) != v for k, v in want.items()):
        return None
    return rec.get("dram_bytes_per_launch")


def _dist():
    from paper_2106_07927_gb300 import replicas
    return replicas.env()


def _cpu_info():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count()


def _oracle_band(left, right, prm, rows):
    import oracle
    t = time.perf_counter()
    oracle.sgm(left[:rows], right[:rows], prm["max_disp"], prm["census_w"], prm["census_h"],
               prm["p1"], prm["p2"], prm["num_paths"], prm["flags"], prm["lr_threshold"])
    return time.perf_counter() - t


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2106_07927_gb300 import scenes
    left, right, _, prm = scenes.single_pair(WORKLOAD, 0)
    rows = 96
    de = prm["width"] * rows * prm["max_disp"]
    for _ in range(args.warmup):
        _oracle_band(left, right, prm, rows)
    times = [_oracle_band(left, right, prm, rows) for _ in range(args.steps)]
    t = sum(times)
    value = de * args.steps / t / 1e6
    model, ncpu = _cpu_info()
    sample = f"{prm['width']}x{rows} band (rows 0..{rows - 1}) of the 1242x375 pair, D=128"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MDE/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16/int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": "MDE/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": model, "host_cores": ncpu},
        "e2e": {"value": round(value, 3), "unit": "MDE/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed work runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=10)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sms.append(float(f[0]))
                maxes.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes),
                "reasons": sorted(reasons), "samples": len(sms)}


def _batch_inputs(n, torch):
    """64 uneven pairs: W, H, D drawn as listed, textures cropped from one generated scene per
    (kind, D) so the inputs take seconds to make."""
    from paper_2106_07927_gb300 import scenes
    specs = scenes.batch_specs(0, n)
    masters = {}
    out = []
    for s in specs:
        p = s["prm"]
        key = (s["kind"], p["max_disp"])
        if key not in masters:
            masters[key] = scenes.make_scene(s["kind"], 17 + len(masters), 1920, 1080,
                                             p["max_disp"])
        L, R, _ = masters[key]
        W, H, D = p["width"], p["height"], p["max_disp"]
        out.append((torch.from_numpy(L[:H, :W].copy()).cuda(),
                    torch.from_numpy(R[:H, :W].copy()).cuda(), W, H, D))
    return out


def _serving_sweep(args, torch, np):
    """Continuous batching over 4 streams (serve.Server): the same 10,000 requests (sizes of the
    batch workload plus 5 % 3840x2160 with D = 256, Poisson arrivals) at each arrival rate;
    latency = completion - arrival. A 1 % sample (the same requests at every rate) must give the
    same map at every rate and equal the CPU oracle (checked after the sweep, off the clock)."""
    import concurrent.futures

    import oracle
    from paper_2106_07927_gb300 import binding, serve
    srv = serve.Server(n_streams=4, max_batch=16)
    rates = [float(r) for r in args.serve_rates.split(",")]
    n = args.serve_requests
    idx = sorted(np.random.default_rng(1).choice(n, max(1, n // 100), replace=False).tolist())
    pool, per_rate, first, same, launches = None, [], None, True, 0
    for rate in rates:
        reqs, pool = serve.make_requests(torch, n, rate, 0, 0.05, pool)
        warm, _ = serve.make_requests(torch, 32, rate, 1, 0.05, pool)
        srv.run(warm)
        l0 = srv.launches
        st = srv.run(reqs)
        st["rate_per_s"] = rate
        st["gpu_launches"] = srv.launches - l0
        launches += st["gpu_launches"]
        served_per_s = st["served"] / max(st["span_s"], 1e-9)
        st["served_pairs_per_s"] = round(served_per_s, 1)
        st["keeps_up"] = bool(served_per_s >= 0.95 * rate)
        outs = {i: binding.u16(reqs[i].out) for i in idx}
        if first is None:
            first = (outs, {i: (reqs[i].left.cpu().numpy(), reqs[i].right.cpu().numpy(),
                                reqs[i].D) for i in idx})
        else:
            same = same and all(np.array_equal(outs[i], first[0][i]) for i in idx)
        per_rate.append(st)
        del reqs
    srv.close()
    # the sample against the oracle (single-threaded C per pair, pairs in parallel threads: the
    # oracle's ctypes calls release the GIL)
    oracle._load()
    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        futs = {i: ex.submit(oracle.sgm, L, R, D, 9, 7, 10, 120, 8, 3)
                for i, (L, R, D) in first[1].items()}
        mism = sum(not np.array_equal(first[0][i], f.result()) for i, f in futs.items())
    kept = [p["rate_per_s"] for p in per_rate if p["keeps_up"]]
    return {"per_rate": per_rate, "streams": 4, "max_batch": 16, "requests_per_rate": n,
            "max_sustained_rate_per_s": max(kept) if kept else None,
            "sample_checked_vs_oracle": len(idx), "sample_mismatches_vs_oracle": int(mism),
            "sample_same_at_every_rate": bool(same), "gpu_launches": launches,
            "sizes": "as the batch, plus 5 % 3840x2160 with D = 256",
            "keeps_up": "served pairs/s >= 0.95 x the arrival rate"}


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = _dist()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_07927_gb300 import binding, scenes

    from paper_2106_07927_gb300 import replicas
    max_over_ranks = replicas.max_over_ranks

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    left, right, prm, workload = _workload_pair(args, 0)
    W, H, D = prm["width"], prm["height"], prm["max_disp"]
    de = W * H * D
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = binding.Stereo(prm)
    Ld = torch.from_numpy(left).cuda()
    Rd = torch.from_numpy(right).cuda()
    out = torch.empty((H, W), dtype=torch.int16, device="cuda")
    if args.profile_steps > 0:  # a bare run of plain steps for a profiler, no timing
        if args.cost_mode:
            t = binding.res2tac_get_tuning(ctx.handle)
            t.cost_mode = args.cost_mode
            binding.res2tac_set_tuning(ctx.handle, t)
        pair = binding.res2tac_pair(Ld.data_ptr(), Rd.data_ptr(), W, out.data_ptr(), 2 * W, W,
                                    H, D, 0)
        for _ in range(args.profile_steps):
            if args.profile_batch:
                binding.res2tac_compute_batch(ctx.handle, [pair], sh)
            binding.res2tac_compute(ctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, out.data_ptr(),
                                    2 * W, sh)
        torch.cuda.synchronize()
        ctx.close()
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    int_peak = binding.res2tac_probe_int_peak(2000, sh)  # lane-ops/s, packed u16 min + add
    popc_rate = binding.res2tac_probe_popc_rate(2000, sh)  # 32-bit POPC per second
    # bytes/s of TMA bulk add-reductions into a buffer the size of the aggregated volume
    red_peak = binding.res2tac_probe_red_peak(2 * W * H * D, 16, sh)

    def step():
        binding.res2tac_compute(ctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, out.data_ptr(),
                                2 * W, sh)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = {k: 0.0 for k in binding.STAGES}
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        launches = binding.res2tac_last_launch_count(ctx.handle) * args.steps

        # per-stage times, in a separate profiled pass (events between the stages)
        binding.res2tac_set_profiling(ctx.handle, True)
        for i in range(args.steps):
            flush.zero_()
            step()
            st = binding.res2tac_stage_times(ctx.handle)  # waits for this step's events
            for k, v in st.items():
                stage[k] += v

        def time_variant(handle, step_fn):
            """Mean device ms of step_fn over the timed steps (same flush and events as the
            plain step), then the stage times of one more profiled pass."""
            nonlocal launches
            binding.res2tac_set_profiling(handle, False)
            for _ in range(3):
                flush.zero_()
                step_fn()
            torch.cuda.synchronize()
            barrier()
            for i in range(args.steps):
                flush.zero_()
                ev0[i].record(stream)
                step_fn()
                ev1[i].record(stream)
            barrier()
            torch.cuda.synchronize()
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / args.steps)
            launches += binding.res2tac_last_launch_count(handle) * args.steps
            binding.res2tac_set_profiling(handle, True)
            flush.zero_()
            step_fn()
            st = binding.res2tac_stage_times(handle)
            binding.res2tac_set_profiling(handle, False)
            return ms, {k: round(v, 4) for k, v in st.items()}

        # the same step with sub-pixel refinement ("fine", Sec. 2.1.3): float map out
        outf = torch.empty((H, W), dtype=torch.float32, device="cuda")
        sub_ms, sub_st = time_variant(ctx.handle, lambda: binding.res2tac_compute_subpixel(
            ctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, outf.data_ptr(), 4 * W, sh))
        fo = outf.cpu().numpy()
        io = binding.u16(out)
        inv = io == binding.RES2TAC_INVALID
        subpixel = {
            "value": round(ws * de / (sub_ms / 1e3) / 1e6, 1), "unit": "MDE/s",
            "ms_per_step": round(sub_ms, 4), "stage_ms": sub_st,
            "same_validity_as_integer_map": bool(np.array_equal(np.isinf(fo), inv)),
            "max_abs_diff_to_integer_map": float(np.abs(fo[~inv] - io[~inv]).max())
            if (~inv).any() else 0.0,
        }

        def variant(flags, **over):
            vctx = binding.Stereo(dict(prm, flags=prm["flags"] | flags, **over))
            o = torch.empty((H, W), dtype=torch.int16, device="cuda")
            ms, st = time_variant(vctx.handle, lambda: binding.res2tac_compute(
                vctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, o.data_ptr(), 2 * W, sh))
            res = binding.u16(o)
            vctx.close()
            return {"value": round(ws * de / (ms / 1e3) / 1e6, 1), "unit": "MDE/s",
                    "ms_per_step": round(ms, 4), "stage_ms": st,
                    "valid_fraction": round(float((res != binding.RES2TAC_INVALID).mean()), 4)}

        # exact consistency check ("exact-cc", Sec. 3.2.3): D^R from a second full matching of
        # the swapped, flipped pair
        exact_cc = variant(binding.RES2TAC_EXACT_CC)
        exact_cc["valid_fraction_approximate_check"] = round(
            float((binding.u16(out) != binding.RES2TAC_INVALID).mean()), 4)
        # the same step with the cost volume computed on the tensor cores (tuning cost_mode 2:
        # a dot product over the census bits, tcgen05): its timing and bit-identity of the map
        tensor_cost = None
        if prm["census_w"] == 9 and D in (64, 128):
            tctx = binding.Stereo(prm)
            t = binding.res2tac_get_tuning(tctx.handle)
            t.cost_mode = 2
            binding.res2tac_set_tuning(tctx.handle, t)
            o = torch.empty((H, W), dtype=torch.int16, device="cuda")
            ms, st = time_variant(tctx.handle, lambda: binding.res2tac_compute(
                tctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, o.data_ptr(), 2 * W, sh))
            tensor_cost = {"value": round(ws * de / (ms / 1e3) / 1e6, 1), "unit": "MDE/s",
                           "ms_per_step": round(ms, 4), "stage_ms": st,
                           "bit_identical_to_default": bool(torch.equal(o, out))}
            tctx.close()
        # the same step with the row-path kernel recomputing its costs from the census
        # descriptors (tuning row_cost 2) instead of reading the cost volume
        row_recompute = None
        if prm["census_w"] in (5, 9) and D % 32 == 0 and D <= 256:
            rctx = binding.Stereo(prm)
            t = binding.res2tac_get_tuning(rctx.handle)
            t.agg_dpl, t.row_mode, t.row_cost = D // 32, 2, 2
            binding.res2tac_set_tuning(rctx.handle, t)
            o = torch.empty((H, W), dtype=torch.int16, device="cuda")
            ms, st = time_variant(rctx.handle, lambda: binding.res2tac_compute(
                rctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, o.data_ptr(), 2 * W, sh))
            row_recompute = {"value": round(ws * de / (ms / 1e3) / 1e6, 1), "unit": "MDE/s",
                             "ms_per_step": round(ms, 4), "stage_ms": st,
                             "bit_identical_to_default": bool(torch.equal(o, out))}
            rctx.close()
        # rectification of the raw pair (Sec. 2.1.1) in front of the same step, through seeded
        # calibration-like maps kept in the context
        rmaps = [torch.from_numpy(m).cuda() for sd in (10, 11)
                 for m in scenes.rectification_maps(sd, W, H)]
        binding.res2tac_set_rectification(ctx.handle, *[m.data_ptr() for m in rmaps], 4 * W, W, H,
                                          sh)
        outr = torch.empty((H, W), dtype=torch.int16, device="cuda")  # keeps `out` for e2e
        raw_ms, raw_st = time_variant(ctx.handle, lambda: binding.res2tac_compute_raw(
            ctx.handle, Ld.data_ptr(), Rd.data_ptr(), W, outr.data_ptr(), 2 * W, sh))
        rect_only = torch.empty((2, H, W), dtype=torch.uint8, device="cuda")
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(args.steps):
            for i, (img, mx, my) in enumerate(((Ld, rmaps[0], rmaps[1]), (Rd, rmaps[2], rmaps[3]))):
                binding.res2tac_rectify(img.data_ptr(), W, W, H, mx.data_ptr(), my.data_ptr(),
                                        4 * W, rect_only[i].data_ptr(), W, W, H, sh)
        r1.record(stream)
        torch.cuda.synchronize()
        launches += 2 * args.steps
        rectify = {"value": round(ws * de / (raw_ms / 1e3) / 1e6, 1), "unit": "MDE/s",
                   "ms_per_step": round(raw_ms, 4), "stage_ms": raw_st,
                   "rectify_ms_per_pair": round(r0.elapsed_time(r1) / args.steps, 4),
                   "maps": "seeded rotation <= 1 deg, shift <= 1.5 px, radial |k1| <= 0.08"}

        # NCC matching cost (Sec. 2.2.1), 5 x 5 and 9 x 9 patches, the paper's NCC penalties
        ncc = {f"{n}x{n}": variant(binding.RES2TAC_NCC, census_w=n, census_h=n, p1=90, p2=880)
               for n in (5, 9)}

        # end to end through the host-buffer entry point (pinned memory): four distinct pairs of
        # the workload in turn, L2 flushed before every step (outside the step's clock), each
        # step timed on the host from the call to the map in host memory. Two forms: the
        # library's host entry (kernels read the pinned images and write the map in place over
        # NVLink-C2C) and staged copies (one cudaMemcpyAsync per image and for the map around
        # res2tac_compute).
        e2e_pairs = []
        for sd in range(4):
            l_, r_, _, _ = _workload_pair(args, sd)
            e2e_pairs.append((torch.from_numpy(l_).pin_memory(), torch.from_numpy(r_).pin_memory(),
                              torch.empty((H, W), dtype=torch.int16).pin_memory()))
        dL = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        dR = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        dO = torch.empty((H, W), dtype=torch.int16, device="cuda")
        binding.res2tac_set_profiling(ctx.handle, False)

        def host_entry(k):
            hl, hr, ho = e2e_pairs[k]
            binding.res2tac_compute_host(ctx.handle, hl.data_ptr(), hr.data_ptr(), W,
                                         ho.data_ptr(), 2 * W, sh)

        def staged(k):
            hl, hr, ho = e2e_pairs[k]
            dL.copy_(hl, non_blocking=True)
            dR.copy_(hr, non_blocking=True)
            binding.res2tac_compute(ctx.handle, dL.data_ptr(), dR.data_ptr(), W, dO.data_ptr(),
                                    2 * W, sh)
            ho.copy_(dO, non_blocking=True)
            stream.synchronize()

        def e2e_time(fn):
            nonlocal launches
            for i in range(3):
                fn(i % 4)
            barrier()
            tot = 0.0
            for i in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn(i % 4)
                tot += time.perf_counter() - t0
            launches += binding.res2tac_last_launch_count(ctx.handle) * args.steps
            return max_over_ranks(tot)

        e2e_s = e2e_time(host_entry)
        e2e_ok = np.array_equal(e2e_pairs[0][2].numpy().view(np.uint16), binding.u16(out))
        e2e_staged_s = e2e_time(staged)
        e2e_ok = e2e_ok and np.array_equal(e2e_pairs[0][2].numpy().view(np.uint16),
                                           binding.u16(out))

        batched = None
        if not args.no_batch:
            def batch_vs_per_pair(pairs_in):
                """The pairs as one res2tac_compute_batch (autotuned first) and as per-pair
                res2tac_compute launches: MDE/s of both, bit-identity of the maps."""
                nonlocal launches
                bprm = scenes.params(64, 64, 64, 9, 7, 10, 120, 8,
                                     scenes.FLAG_LR_CHECK | scenes.FLAG_MEDIAN)
                bctx = binding.Stereo(bprm)
                bouts, bpairs, singles = [], [], []
                for Lb, Rb, w, h, d in pairs_in:
                    o = torch.empty((h, w), dtype=torch.int16, device="cuda")
                    bouts.append(o)
                    bpairs.append(binding.res2tac_pair(Lb.data_ptr(), Rb.data_ptr(), w,
                                                       o.data_ptr(), 2 * w, w, h, d, 0))
                bde = sum(w * h * d for _, _, w, h, d in pairs_in)
                # the batch autotuner (per bucket of D and size class) before the timed batches
                table, ms_def, ms_tuned = binding.res2tac_autotune_batch(bctx.handle, bpairs, sh)
                for _ in range(2):
                    binding.res2tac_compute_batch(bctx.handle, bpairs, sh)
                torch.cuda.synchronize()
                be0 = torch.cuda.Event(enable_timing=True)
                be1 = torch.cuda.Event(enable_timing=True)
                barrier()
                be0.record(stream)
                for _ in range(args.batch_steps):
                    binding.res2tac_compute_batch(bctx.handle, bpairs, sh)
                be1.record(stream)
                barrier()
                t_batch = max_over_ranks(be0.elapsed_time(be1) / 1e3 / args.batch_steps)
                launches += binding.res2tac_last_launch_count(bctx.handle) * args.batch_steps
                batch_result = [o.clone() for o in bouts]
                # the same pairs as per-pair launches, one context each
                souts = []
                for Lb, Rb, w, h, d in pairs_in:
                    c = binding.Stereo(scenes.params(w, h, d, 9, 7, 10, 120, 8, 3))
                    singles.append((c, Lb, Rb, w, h))
                    souts.append(torch.empty((h, w), dtype=torch.int16, device="cuda"))

                def per_pair():
                    for (c, Lb, Rb, w, h), o in zip(singles, souts):
                        binding.res2tac_compute(c.handle, Lb.data_ptr(), Rb.data_ptr(), w,
                                                o.data_ptr(), 2 * w, sh)

                per_pair()
                torch.cuda.synchronize()
                barrier()
                be0.record(stream)
                for _ in range(args.batch_steps):
                    per_pair()
                be1.record(stream)
                barrier()
                t_single = max_over_ranks(be0.elapsed_time(be1) / 1e3 / args.batch_steps)
                launches += sum(binding.res2tac_last_launch_count(c.handle)
                                for c, *_ in singles) * args.batch_steps
                same = all(torch.equal(a, b) for a, b in zip(batch_result, souts))
                for c, *_ in singles:
                    c.close()
                bctx.close()
                return {
                    "value": round(ws * bde / t_batch / 1e6, 1), "unit": "MDE/s",
                    "pairs": len(pairs_in), "de_per_batch": bde,
                    "ms_per_batch": round(1e3 * t_batch, 3),
                    "per_pair_launches": {"value": round(ws * bde / t_single / 1e6, 1),
                                          "ms_per_batch": round(1e3 * t_single, 3)},
                    "speedup_vs_per_pair": round(t_single / t_batch, 3),
                    "bit_identical_to_per_pair": bool(same),
                    "autotune": {"table": [e.as_dict() for e in table],
                                 "mde_per_s_default": round(bde / (ms_def / 1e3) / 1e6, 1),
                                 "mde_per_s_tuned": round(bde / (ms_tuned / 1e3) / 1e6, 1),
                                 "ms_default": round(ms_def, 3), "ms_tuned": round(ms_tuned, 3)}}

            batched = batch_vs_per_pair(_batch_inputs(args.batch_pairs, torch))
            batched["sizes"] = ("W in {320,640,1024,1242,1920}, H in {240,375,512,768,1080}, "
                                "D in {64,128,256}, seed 0")
            # batches of one size: the 1242x375 D=128 pair (16 seeded pairs) and the 320x240
            # D=64 pair of the small workload (64 pairs), census 9x7 as in the mix
            same_size = {}
            for name, n, wl in (("1242x375_d128 x16", 16, WORKLOAD),
                                ("320x240_d64 x64", 64, "320x240_d64_ct5x5_r4")):
                items = []
                for sd in range(n):
                    l_, r_, _, p_ = scenes.single_pair(wl, sd)
                    items.append((torch.from_numpy(l_).cuda(), torch.from_numpy(r_).cuda(),
                                  p_["width"], p_["height"], p_["max_disp"]))
                same_size[name] = batch_vs_per_pair(items)
            batched["same_size_batches"] = same_size
        serving = None
        if not args.no_serve and rank == 0:
            serving = _serving_sweep(args, torch, np)
    mean_ms = max_over_ranks(sum(step_ms) / len(step_ms))
    value = ws * de / (mean_ms / 1e3) / 1e6
    subpixel["throughput_vs_integer_step"] = round(mean_ms / subpixel["ms_per_step"], 3)
    exact_cc["throughput_vs_integer_step"] = round(mean_ms / exact_cc["ms_per_step"], 3)
    for v in ncc.values():
        v["throughput_vs_census_step"] = round(mean_ms / v["ms_per_step"], 3)
    rectify["throughput_vs_rectified_input"] = round(mean_ms / rectify["ms_per_step"], 3)
    agg_ms = stage["aggregate"] / args.steps
    # algorithmic operations and bytes of the aggregation per launch (16-bit lane operations):
    # 9 per DE and path (8 of the recurrence, 1 accumulation) + 2 per DE (cost xor/popcount read)
    ops_agg = de * (9 * prm["num_paths"] + 2)
    bytes_agg = 2 * de + 16 * W * H
    achieved = ops_agg / (agg_ms / 1e3)
    hbm = peaks.get("hbm_gbs")
    dominant = max(stage, key=stage.get)
    clocks = clk.summary()
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "MDE/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8/u16 (integer)", "data": "synthetic",
        "config": {"workload": workload, "W": W, "H": H, "D": D, "census": "9x7", "paths": 8,
                   "P1": 10, "P2": 120, "post": "LR check (1 px) + 3x3 median",
                   "l2": "flushed between steps (256 MB write outside the step events)",
                   "parallelism": f"replicas x{ws}"},
        "fps": round(1e3 / mean_ms * ws, 1),
        "stage_ms": {k: round(v / args.steps, 4) for k, v in stage.items()},
        "subpixel": subpixel,
        "exact_cc": exact_cc,
        "tensor_core_cost": tensor_cost,
        "row_recompute": row_recompute,
        "ncc": ncc,
        "rectify": rectify,
        "roofline": {"kernel": "aggregate (SGM paths)", "bound": "alu",
                     "achieved": round(achieved / 1e12, 3),
                     "peak": round(int_peak / 1e12, 3), "unit": "T lane-ops/s",
                     "frac": round(achieved / int_peak, 3),
                     "peak_source": "measured packed-u16 min+add probe on this GPU",
                     "hbm_achieved_gbs": round(bytes_agg / (agg_ms / 1e3) / 1e9, 1),
                     "hbm_peak_gbs": hbm,
                     "traffic": (_traffic(binding.res2tac_get_tuning(ctx.handle))
                                 if args.pair is None else None),
                     "ops_per_launch": ops_agg, "algorithmic_bytes_per_launch": bytes_agg,
                     "dominant_stage": dominant,
                     # the accumulation into S: every path adds 2 bytes per DE (read-modify-write
                     # in L2), against the measured rate of bulk add-reductions
                     "s_accumulation": {
                         "bytes_per_launch": 2 * de * prm["num_paths"],
                         "achieved_gbs": round(2 * de * prm["num_paths"] / (agg_ms / 1e3) / 1e9, 1),
                         "peak_gbs": round(red_peak / 1e9, 1),
                         "frac": round(2 * de * prm["num_paths"] / (agg_ms / 1e3) / red_peak, 3),
                         "peak_source": "measured TMA bulk add-reduction probe, S-sized buffer"}},
        # recomputing the cost inside each path walk instead of reading the volume: two 32-bit
        # POPC per DE and path at the measured POPC rate, against the aggregation's own time
        "cost_recompute_bound": {
            "popc_per_s": round(popc_rate, 0),
            "popc_per_step": 2 * prm["num_paths"] * de,
            "popc_us_per_step": round(2 * prm["num_paths"] * de / popc_rate * 1e6, 1),
            "aggregate_us_per_step": round(agg_ms * 1e3, 1),
            "cost_bytes_read_per_step": prm["num_paths"] * de},
        "e2e": {"value": round(ws * de * args.steps / e2e_s / 1e6, 1), "unit": "MDE/s",
                "h2d_bytes_per_step": 2 * W * H, "d2h_bytes_per_step": 2 * W * H,
                "ms_per_step": round(1e3 * e2e_s / args.steps, 4), "matches_device_path": e2e_ok,
                "api": "res2tac_compute_host (pinned buffers read and written in place)",
                "inputs": "4 distinct pairs in turn, L2 flushed before every step",
                "staged_copies": {
                    "value": round(ws * de * args.steps / e2e_staged_s / 1e6, 1),
                    "ms_per_step": round(1e3 * e2e_staged_s / args.steps, 4),
                    "api": "cudaMemcpyAsync per image + res2tac_compute + cudaMemcpyAsync of the "
                           "map"}},
        "batched": batched,
        "serving": serving,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed_plain": round(t_wall, 3),
    }
    if rank == 0 and not args.no_cpu and args.pair is None:
        t = [_oracle_band(left, right, prm, H) for _ in range(3)]
        model, ncpu = _cpu_info()
        result["cpu_baseline"] = {
            "value": round(de / statistics.median(t) / 1e6, 3), "unit": "MDE/s", "cores": 1,
            "kind": "oracle", "sample": "the full 1242x375 D=128 pair, 3 runs, median",
            "cpu": model, "host_cores": ncpu}
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
