"""Continuous-batching serving loop over the C ABI (the paper has no serving mode; this is the
library's own addition).

Requests (stereo pairs of uneven W, H, D) arrive as a Poisson process. The server keeps S CUDA
streams, each with its own context whose batch engine is reserved once (res2tac_batch_reserve),
so nothing is allocated while serving and the per-stream method parameters stay resident on the
device. Whenever a stream is idle, it admits the waiting requests in arrival order while their
device memory (res2tac_batch_workspace_bytes: cost and aggregated volumes, maps) fits
the stream's reservation, and runs them as one res2tac_compute_batch. Requests that arrive while
others are on the GPU join the next batch of the next free stream; batches on different streams
overlap on the device. Latency is completion (host time at which the stream's event is observed
complete) minus arrival.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import binding, scenes


class Request:
    """One stereo pair to serve. status: "waiting", then "ok", "cancelled" (cancel() called before
    the request was admitted; it never reaches the GPU) or "failed: <message>" (its batch was
    refused by the library; the server carries on with the next batches)."""
    __slots__ = ("idx", "arrival", "W", "H", "D", "left", "right", "out", "done", "stream",
                 "batch_size", "need", "status")

    def __init__(self, idx, arrival, left, right, W, H, D):
        self.idx, self.arrival = idx, arrival
        self.left, self.right = left, right
        self.W, self.H, self.D = W, H, D
        self.out = None
        self.done = None
        self.stream = None
        self.batch_size = 0
        self.need = 0
        self.status = "waiting"

    def cancel(self):
        if self.status == "waiting":
            self.status = "cancelled"


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


class Server:
    def __init__(self, census=(9, 7), p1=10, p2=120, num_paths=8,
                 flags=scenes.FLAG_LR_CHECK | scenes.FLAG_MEDIAN, n_streams=4, max_batch=16,
                 budget_bytes=None):
        import torch
        self.torch = torch
        self.method = dict(census_w=census[0], census_h=census[1], p1=p1, p2=p2,
                           num_paths=num_paths, flags=flags, lr_threshold=1)
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        prm = scenes.params(64, 64, 64, census[0], census[1], p1, p2, num_paths, flags)
        self.params = binding.params_from_dict(prm)
        self.ctx = [binding.Stereo(prm) for _ in range(n_streams)]
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(min(0.6 * free, 96e9))
        self.per_stream = budget_bytes // n_streams
        for c in self.ctx:
            binding.res2tac_batch_reserve(c.handle, self.per_stream, max_batch)
        self.launches = 0

    def need_bytes(self, W, H, D) -> int:
        pair = binding.res2tac_pair(None, None, W, None, 2 * W, W, H, D, 0)
        return binding.res2tac_batch_workspace_bytes(self.params, [pair])

    def close(self):
        for c in self.ctx:
            c.close()
        self.ctx = []

    def _launch(self, slot, batch):
        torch = self.torch
        st = self.streams[slot]
        pairs = []
        with torch.cuda.stream(st):
            for r in batch:
                r.out = torch.empty((r.H, r.W), dtype=torch.int16, device="cuda")
                pairs.append(binding.res2tac_pair(r.left.data_ptr(), r.right.data_ptr(),
                                                  r.left.stride(0), r.out.data_ptr(), 2 * r.W,
                                                  r.W, r.H, r.D, 0))
                r.stream = slot
                r.batch_size = len(batch)
        try:
            binding.res2tac_compute_batch(self.ctx[slot].handle, pairs, st.cuda_stream)
        except binding.Res2tacError as e:  # refused on the host: nothing was launched
            for r in batch:
                r.status = f"failed: {e}"
                r.out = None
            return None
        self.launches += binding.res2tac_last_launch_count(self.ctx[slot].handle)
        ev = torch.cuda.Event()
        ev.record(st)
        return ev

    def run(self, requests):
        """Serves the requests (sorted by arrival, seconds from the start) in real time."""
        n = len(requests)
        for r in requests:
            r.need = self.need_bytes(r.W, r.H, r.D)
            if r.need > self.per_stream:
                raise ValueError(f"request {r.idx} needs {r.need} B > stream budget "
                                 f"{self.per_stream} B")
        pending = collections.deque()
        inflight = {}
        free_slots = list(range(len(self.streams)))[::-1]
        i = done = 0
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            while i < n and requests[i].arrival <= now:
                pending.append(requests[i])
                i += 1
            for slot in list(inflight):
                ev, batch = inflight[slot]
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in batch:
                        r.done = tdone
                        r.status = "ok"
                    done += len(batch)
                    del inflight[slot]
                    free_slots.append(slot)
            while pending and pending[0].status == "cancelled":  # dropped before admission
                pending.popleft().done = time.perf_counter() - t0
                done += 1
            while free_slots and pending:
                batch, mem = [], 0
                while pending and len(batch) < self.max_batch and \
                        mem + pending[0].need <= self.per_stream:
                    r = pending.popleft()
                    if r.status == "cancelled":
                        r.done = time.perf_counter() - t0
                        done += 1
                        continue
                    batch.append(r)
                    mem += r.need
                if not batch:
                    continue
                slot = free_slots.pop()
                ev = self._launch(slot, batch)
                if ev is None:  # the batch failed: its requests are done, the stream is free
                    tdone = time.perf_counter() - t0
                    for r in batch:
                        r.done = tdone
                    done += len(batch)
                    free_slots.append(slot)
                else:
                    inflight[slot] = (ev, batch)
        self.torch.cuda.synchronize()
        return summarize(requests)


def summarize(requests):
    """Throughput and latency over the requests served ("ok"); counts of the others."""
    ok = [r for r in requests if r.status == "ok"] or requests[:1]
    lat = np.array([r.done - r.arrival for r in ok]) * 1e3
    de = sum(r.W * r.H * r.D for r in ok)
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    return {
        "requests": len(requests),
        "served": sum(r.status == "ok" for r in requests),
        "cancelled": sum(r.status == "cancelled" for r in requests),
        "failed": sum(r.status.startswith("failed") for r in requests),
        "mde_per_s": round(de / max(span, 1e-9) / 1e6, 1),
        "p50_ms": round(float(np.percentile(lat, 50)), 3),
        "p99_ms": round(float(np.percentile(lat, 99)), 3),
        "p999_ms": round(float(np.percentile(lat, 99.9)), 3),
        "mean_batch": round(float(np.mean([r.batch_size for r in ok])), 2),
        "span_s": round(span, 3),
    }


class ScenePool:
    """Device-resident inputs of every requested shape, cropped from one generated 1920x1080 scene
    per kind (disparities for D = 256). Pairs larger than that are cropped from the same scene
    upsampled 2x in both axes, which is again a rectified pair, with twice the disparities."""

    def __init__(self, torch, seed=0, master=(1920, 1080)):
        self.torch, self.seed, self.master = torch, seed, master
        self.masters, self.cache = {}, {}

    def _master(self, kind, big):
        key = (kind, big)
        if key not in self.masters:
            if big:
                L, R = self._master(kind, False)
                up = lambda a: np.repeat(np.repeat(a, 2, axis=0), 2, axis=1)
                self.masters[key] = (up(L), up(R))
            else:
                L, R, _ = scenes.make_scene(kind, self.seed + 97 * len(self.masters),
                                            self.master[0], self.master[1], 256)
                self.masters[key] = (L, R)
        return self.masters[key]

    def get(self, kind, W, H, D):
        key = (kind, W, H, D)
        if key not in self.cache:
            big = W > self.master[0] or H > self.master[1]
            L, R = self._master(kind, big)
            t = self.torch
            self.cache[key] = (t.from_numpy(L[:H, :W].copy()).cuda(),
                               t.from_numpy(R[:H, :W].copy()).cuda())
        return self.cache[key]


def make_requests(torch, n, rate, seed=0, big_fraction=0.05, pool=None):
    specs = scenes.batch_specs(seed, n, big_fraction)
    arrivals = poisson_arrivals(n, rate, seed)
    pool = pool or ScenePool(torch, seed)
    reqs = []
    for i, (s, t) in enumerate(zip(specs, arrivals)):
        p = s["prm"]
        L, R = pool.get(s["kind"], p["width"], p["height"], p["max_disp"])
        reqs.append(Request(i, float(t), L, R, p["width"], p["height"], p["max_disp"]))
    return reqs, pool


def check_alone(server, requests, sample_idx):
    """Recomputes sampled requests alone (one res2tac_compute each) and compares bit-exactly."""
    torch = server.torch
    bad = []
    for i in sample_idx:
        r = requests[i]
        c = binding.Stereo(scenes.params(r.W, r.H, r.D, server.method["census_w"],
                                         server.method["census_h"], server.method["p1"],
                                         server.method["p2"], server.method["num_paths"],
                                         server.method["flags"]))
        alone = c.compute(r.left, r.right)
        torch.cuda.synchronize()
        if not torch.equal(alone, r.out):
            bad.append(i)
        c.close()
    return bad


def main():
    import argparse
    import json

    import torch
    ap = argparse.ArgumentParser(description="serving sweep over arrival rates")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--rates", default="200,500,1000,2000,5000")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--big-fraction", type=float, default=0.05)
    ap.add_argument("--sample", type=float, default=0.01)
    args = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    srv = Server(n_streams=args.streams, max_batch=args.max_batch)
    pool = None
    for rate in [float(x) for x in args.rates.split(",")]:
        reqs, pool = make_requests(torch, args.requests, rate, 0, args.big_fraction, pool)
        warm, _ = make_requests(torch, 32, rate, 1, args.big_fraction, pool)
        srv.run(warm)
        stats = srv.run(reqs)
        rng = np.random.default_rng(1)
        idx = sorted(rng.choice(len(reqs), max(1, int(args.sample * len(reqs))), replace=False))
        stats["sample_alone_mismatches"] = len(check_alone(srv, reqs, idx))
        stats["sample_checked"] = len(idx)
        stats["rate_per_s"] = rate
        print(json.dumps(stats), flush=True)
    srv.close()


if __name__ == "__main__":
    main()
