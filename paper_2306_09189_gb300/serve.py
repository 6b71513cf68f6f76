"""Continuous-batching serving loop for encrypted images of mixed resolutions.

A stack of 4 x [conv3x3 + folded BatchNorm, Chebyshev GELU, 2x2 average pool] (the layer
programs of Sec. 4 and the activation of the Appendix) is planned once per input resolution on
a root context: rotation keys, diagonal and mask plaintexts stay resident in HBM.  Two servers:

* BatchServer (the default): continuous batching at stage granularity on one stream.  Admitted
  requests wait at their next (resolution, layer); each step runs one such stage for all
  requests waiting there as one batched launch set, so every key and plaintext word is read
  once per group; requests arriving meanwhile are admitted between steps when a slot of their
  resolution is free and HBM headroom allows, and join the next step of their stage.
* Server: one request per worker slot, a slot being a forked context (he_ctx_fork: shares every
  key and table, owns its key-switching scratch) with forked layer objects and its own CUDA
  stream; requests overlap on the device through their streams.

Each request's result is independent of what else runs: the batched calls give every image its
own bits, and a slot's arithmetic touches only its own buffers and the shared read-only keys
and plaintexts.

All homomorphic work runs in libhegpu.so; this module only schedules.
"""
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hegpu as H
from . import host


def poly_depth(deg):
    """Levels of the GELU as the serving loop evaluates it (Paterson-Stockmeyer)."""
    return host.ps_depth(deg)


@dataclass
class Stage:
    conv: object
    pool: object
    lay_in: object
    lay_conv: object
    lay_pool: object
    lv_in: int
    lv_conv: int
    lv_gelu: int
    lv_pool: int


class Stack:
    """The layer programs for one input resolution, planned on the root context."""

    def __init__(self, ctx, m, layers, cheb, level, scale, channels=4, conv_form="diag"):
        self.ctx, self.m, self.cheb, self.scale = ctx, m, np.asarray(cheb, dtype=np.float64), scale
        info = H.he_ctx_info(ctx)
        self.n, self.N = info["n"], info["slots"]
        lay = H.he_layout_image(channels, m, self.N)
        self.in_layout, self.in_level = lay, level
        self.stages = []
        lv = level
        depth = poly_depth(len(cheb) - 1)
        for (W, b) in layers:
            if conv_form == "bsgs":                 # giant stride from the library's cost model
                conv = H.he_conv_create_bsgs(ctx, lay, W, b, 1, 1, lv, scale, 0)
            else:
                conv = H.he_conv_create(ctx, lay, W, b, 1, 1, lv, scale)
            H.he_keygen_rotations(ctx, H.he_conv_rotations(conv))
            lay_c = H.he_conv_out_layout(conv)
            lv_c = lv - 1
            lv_g = lv_c - depth
            pool = H.he_pool_create(ctx, lay_c, lv_g)
            H.he_keygen_rotations(ctx, H.he_pool_rotations(pool))
            lay_p = H.he_pool_out_layout(pool)
            self.stages.append(Stage(conv, pool, lay, lay_c, lay_p, lv, lv_c, lv_g, lv_g - 2))
            lay, lv = lay_p, lv_g - 2
        self.out_layout, self.out_level = lay, lv

    def destroy(self):
        for st in self.stages:
            H.he_conv_destroy(st.conv)
            H.he_pool_destroy(st.pool)


class Worker:
    """One slot: a forked context, forked layer objects per resolution, its own stream."""

    def __init__(self, root, stacks, device=0):
        import torch
        self.ctx = H.he_ctx_fork(root)
        self.stream = torch.cuda.Stream(device=device)
        self.stacks = stacks
        self.forks = {}
        self.bufs = {}
        for m, st in stacks.items():
            fs = [(H.he_conv_fork(s.conv, self.ctx), H.he_pool_fork(s.pool, self.ctx)) for s in st.stages]
            self.forks[m] = fs
            b = {"in": [H.he_ct_alloc(self.ctx, st.in_level) for _ in range(st.in_layout.n_shards)]}
            for i, s in enumerate(st.stages):
                b["conv%d" % i] = [H.he_ct_alloc(self.ctx, s.lv_conv) for _ in range(s.lay_conv.n_shards)]
                b["pool%d" % i] = [H.he_ct_alloc(self.ctx, s.lv_pool) for _ in range(s.lay_pool.n_shards)]
            self.bufs[m] = b

    def run(self, m, in_coeffs, mode=H.HE_FUSED):
        """Import the encrypted input (coefficient form), run the stack, return output handles."""
        st, fs, b = self.stacks[m], self.forks[m], self.bufs[m]
        s = self.stream
        for ct, co in zip(b["in"], in_coeffs):
            H.he_ct_import_coeffs(ct, co, st.in_level, st.scale, s)
        cur = b["in"]
        for i, (stage, (conv, pool)) in enumerate(zip(st.stages, fs)):
            outc = b["conv%d" % i]
            H.he_conv_run(self.ctx, conv, cur, outc, mode, s)
            if mode == H.HE_PLAIN:
                for ct in outc:
                    H.he_poly_eval(self.ctx, ct, st.cheb, st.scale, s)
            else:                                  # all shards of the layer through the products together
                H.he_poly_eval_ps_many(self.ctx, outc, st.cheb, [st.scale] * len(outc), s)
            outp = b["pool%d" % i]
            H.he_pool_run(self.ctx, pool, outc, outp, mode, s)
            cur = outp
        s.synchronize()
        return cur

    def destroy(self):
        for m, fs in self.forks.items():
            for conv, pool in fs:
                H.he_conv_destroy(conv)
                H.he_pool_destroy(pool)
            for cts in self.bufs[m].values():
                for ct in cts:
                    H.he_ct_free(ct)
        H.he_ctx_destroy(self.ctx)


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    m: int                   # input side
    coeffs: list             # encrypted input shards, coefficient form
    start: float = None
    finish: float = None
    result: list = field(default_factory=list)


class Server:
    """Admits arrivals onto free worker slots while HBM headroom allows; slots run concurrently."""

    def __init__(self, root, stacks, n_workers, reserve_bytes=2 << 30, export=True, workers=None,
                 hbm_free=None, admit_timeout=10.0):
        self.root, self.stacks = root, stacks
        self.admit_timeout = admit_timeout
        self.reserve = reserve_bytes
        self.export = export
        self.workers = workers if workers is not None else [Worker(root, stacks) for _ in range(n_workers)]
        self._free_fn = hbm_free

    def _hbm_free(self):
        if self._free_fn is not None:
            return self._free_fn()
        import torch
        return torch.cuda.mem_get_info()[0]

    def serve(self, requests):
        """Run the requests (arrival times relative to now); returns them with timings."""
        idle = queue.Queue()
        for w in self.workers:
            idle.put(w)
        done = []
        lock = threading.Lock()
        threads = []
        t0 = time.perf_counter()

        def job(w, r):
            r.start = time.perf_counter() - t0
            out = w.run(r.m, r.coeffs)
            if self.export:
                r.result = [H.he_ct_export_coeffs(w.ctx, ct, self.stacks[r.m].n, w.stream) for ct in out]
            else:
                r.result = out
            r.finish = time.perf_counter() - t0
            with lock:
                done.append(r)
            idle.put(w)

        for r in sorted(requests, key=lambda x: x.arrival):
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            w = idle.get()                               # a slot is free
            t_wait = time.perf_counter()
            while self._hbm_free() < self.reserve:       # and memory headroom
                if idle.qsize() == len(self.workers) - 1 and time.perf_counter() - t_wait > self.admit_timeout:
                    # nothing of ours runs to free memory, and nothing else did meanwhile
                    raise MemoryError("serve: HBM headroom below the %d-byte reserve for %.1f s with no "
                                      "request running" % (self.reserve, self.admit_timeout))
                time.sleep(0.001)
            th = threading.Thread(target=job, args=(w, r))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        return sorted(done, key=lambda x: x.rid)

    def destroy(self):
        for w in self.workers:
            w.destroy()


def next_group(waiting, sizes):
    """The next batched step: waiting = [(arrival, rid, m, stage)] of the admitted requests.
    Returns ((m, stage), [rid]): the stage of the request that arrived first, and the oldest
    requests waiting at that stage, as many as the largest group size in `sizes` allows."""
    first = min(waiting)
    key = (first[2], first[3])
    here = sorted(w for w in waiting if (w[2], w[3]) == key)
    size = max(b for b in sizes if b <= len(here))
    return key, [w[1] for w in here[:size]]


class BatchServer:
    """Continuous batching at stage granularity on one stream.

    Admitted requests wait at their next stage (resolution m, layer i).  Every scheduling step
    takes the stage whose oldest waiting request arrived first and runs it for every request
    waiting there (up to max_batch, in a power-of-two group): one he_conv_run_batch, so each
    rotation key and diagonal plaintext is streamed from HBM once for the whole group, then the
    GELU of all their shards in one he_poly_eval_ps_many, then each request's pooling.
    Requests that arrive meanwhile are admitted between steps as soon as a slot of their
    resolution is free and HBM headroom allows, and join the next step of their stage.  Each
    image's result is the one it gets alone (the batched calls give every image exactly its
    own bits).  Slots (per-request buffers) are allocated up front, so admission allocates
    nothing.  With export=False a finished request's result is the handles of its slot, which
    then stays with the request instead of returning to the pool."""

    def __init__(self, root, stacks, max_batch=4, slots_per_res=4, reserve_bytes=2 << 30, export=True,
                 hbm_free=None, key_stream=H.HE_KEY_STREAM_LDG, admit_timeout=10.0):
        import torch
        self.root, self.stacks, self.export = root, stacks, export
        self.admit_timeout = admit_timeout
        self.max_batch, self.reserve, self._free_fn = max_batch, reserve_bytes, hbm_free
        self.stream = torch.cuda.Stream()
        self.sizes = [1 << k for k in range(max_batch.bit_length()) if (1 << k) <= max_batch]
        # one fused launch per (stage, group size) lives at once: the register-fed key stream keeps
        # their memory to the batch buffers (the pre-keyed tables each autotuned launch may take,
        # a quarter of what is free at its turn, add up over many launches)
        self._prev_key_stream = H.he_ctx_get_option(root, H.HE_OPT_KEY_STREAM)
        H.he_ctx_set_option(root, H.HE_OPT_KEY_STREAM, key_stream)
        # one conv object per (stage, group size): each keeps the buffers of its own batch shape
        self.convs = {m: [{b: H.he_conv_fork(stg.conv, root) for b in self.sizes} for stg in st.stages]
                      for m, st in stacks.items()}
        self.free = {m: [] for m in stacks}
        for m, st in stacks.items():
            for _ in range(slots_per_res):
                b = {"in": [H.he_ct_alloc(root, st.in_level) for _ in range(st.in_layout.n_shards)]}
                for i, stg in enumerate(st.stages):
                    b["conv%d" % i] = [H.he_ct_alloc(root, stg.lv_conv) for _ in range(stg.lay_conv.n_shards)]
                    b["pool%d" % i] = [H.he_ct_alloc(root, stg.lv_pool) for _ in range(stg.lay_pool.n_shards)]
                self.free[m].append(b)
        self.steps = []                               # (m, stage, group size) of every step run

    def _hbm_free(self):
        if self._free_fn is not None:
            return self._free_fn()
        import torch
        return torch.cuda.mem_get_info()[0]

    def _run_stage(self, m, i, group):
        st, stg, s = self.stacks[m], self.stacks[m].stages[i], self.stream
        conv = self.convs[m][i][len(group)]
        ins = [ct for r in group for ct in r._cur]
        outc = [ct for r in group for ct in r._slot["conv%d" % i]]
        H.he_conv_run_batch(self.root, conv, ins, outc, len(group), H.HE_FUSED, s)
        H.he_poly_eval_ps_many(self.root, outc, st.cheb, [st.scale] * len(outc), s)
        for r in group:
            H.he_pool_run(self.root, stg.pool, r._slot["conv%d" % i], r._slot["pool%d" % i], H.HE_FUSED, s)
            r._cur = r._slot["pool%d" % i]
            r._stage = i + 1
        s.synchronize()
        self.steps.append((m, i, len(group)))

    def serve(self, requests):
        """Run the requests (arrival times relative to now); returns them with timings."""
        pending = sorted(requests, key=lambda x: x.arrival)
        active, done = [], []
        t_short = None                                # since when headroom has been short, idle
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now and self.free[pending[0].m]:
                if self._hbm_free() < self.reserve:
                    if not active:           # nothing of ours runs to free memory
                        t_short = t_short if t_short is not None else time.perf_counter()
                        if time.perf_counter() - t_short > self.admit_timeout:
                            raise MemoryError("serve: HBM headroom below the %d-byte reserve for %.1f s "
                                              "with no request running" % (self.reserve, self.admit_timeout))
                    break
                t_short = None
                r = pending.pop(0)
                r._slot = self.free[r.m].pop()
                st = self.stacks[r.m]
                for ct, co in zip(r._slot["in"], r.coeffs):
                    H.he_ct_import_coeffs(ct, co, st.in_level, st.scale, self.stream)
                r._cur, r._stage = r._slot["in"], 0
                r.start = time.perf_counter() - t0
                active.append(r)
            if not active:
                time.sleep(max(0.0, min(0.001, pending[0].arrival - now)))
                continue
            key, group = next_group([(r.arrival, r.rid, r.m, r._stage) for r in active], self.sizes)
            by_rid = {r.rid: r for r in active}
            group = [by_rid[rid] for rid in group]
            self._run_stage(key[0], key[1], group)
            for r in group:
                if r._stage == len(self.stacks[r.m].stages):
                    st = self.stacks[r.m]
                    r.result = ([H.he_ct_export_coeffs(self.root, ct, st.n, self.stream) for ct in r._cur]
                                if self.export else list(r._cur))
                    r.finish = time.perf_counter() - t0
                    active.remove(r)
                    if self.export:
                        self.free[r.m].append(r._slot)
                    done.append(r)
        return sorted(done, key=lambda x: x.rid)

    def destroy(self):
        H.he_ctx_set_option(self.root, H.HE_OPT_KEY_STREAM, self._prev_key_stream)
        for m in self.convs:
            for per_stage in self.convs[m]:
                for cv in per_stage.values():
                    H.he_conv_destroy(cv)
            for b in self.free[m]:
                for cts in b.values():
                    for ct in cts:
                        H.he_ct_free(ct)


def latency_stats(reqs):
    lat = np.array([r.finish - r.arrival for r in reqs])
    span = max(r.finish for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "images_per_s": len(reqs) / span, "n": len(reqs)}


def encrypt_request(ctx, stack, img, nonce):
    """Client side: encrypt an image for `stack` and export the shards (coefficient form)."""
    cts = host.encrypt_image(ctx, stack.in_layout, img, stack.in_level, stack.scale, nonce0=nonce)
    out = [H.he_ct_export_coeffs(ctx, ct, stack.n) for ct in cts]
    for ct in cts:
        H.he_ct_free(ct)
    return out


def decrypt_result(ctx, stack, coeffs):
    """Client side: import the result shards and decrypt the output image."""
    cts = []
    for co in coeffs:
        ct = H.he_ct_alloc(ctx, stack.out_level)
        H.he_ct_import_coeffs(ct, co, stack.out_level, stack.scale)
        cts.append(ct)
    img = host.decrypt_image(ctx, stack.out_layout, cts)
    for ct in cts:
        H.he_ct_free(ct)
    return img


def plaintext_stack(img, layers, cheb, pool=True):
    """FP64 reference of the same network (same polynomial, not GELU itself)."""
    import torch
    x = np.asarray(img, dtype=np.float64)
    for (W, b) in layers:
        t = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), padding=1)[0].numpy()
        t = t + b[:, None, None]
        # p(t) = sum c_k T_k(t), t in [-1, 1]
        T0, T1 = np.ones_like(t), t
        y = cheb[0] * T0 + cheb[1] * T1
        for k in range(2, len(cheb)):
            T0, T1 = T1, 2 * t * T1 - T0
            y = y + cheb[k] * T1
        x = torch.nn.functional.avg_pool2d(torch.tensor(y)[None], 2)[0].numpy() if pool else y
    return x


def run_benchmark(args):
    """The serving measurement; args: sizes, widths, rates, requests, conv, server, workers,
    max_batch (the command-line options).  Returns the result line as a dict."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads
    sizes = [int(x) for x in args.sizes.split(",")]
    widths = tuple(int(x) for x in args.widths.split(","))
    pr = host.serving_params(seed=0)
    root = H.he_ctx_create(pr)
    t = time.perf_counter()
    H.he_keygen_relin(root)
    layers = workloads.serving_stack(0, widths=widths, m=32)
    cheb = host.chebyshev_coeffs("gelu", workloads.GELU_DEGREE, -8.0, 8.0)
    level = pr.n_q - 1
    stacks = {m: Stack(root, m, layers, cheb, level, pr.scale, conv_form=args.conv) for m in sizes}
    setup_s = time.perf_counter() - t
    import torch
    mem = {"after_setup_free_gb": torch.cuda.mem_get_info()[0] / 1e9}
    if args.server == "batch":
        server = BatchServer(root, stacks, max_batch=args.max_batch, slots_per_res=args.max_batch)
    else:
        server = Server(root, stacks, args.workers)
    rng = np.random.default_rng(0)
    mix = {32: 0.6, 64: 0.3, 224: 0.1}
    probs = np.array([mix.get(m, 0.1) for m in sizes])
    probs /= probs.sum()

    def make(n, seed):
        r = np.random.default_rng(seed)
        out = []
        for i in range(n):
            m = int(r.choice(sizes, p=probs))
            img = r.uniform(0, 1, (4, m, m))
            img[3] = 0.0
            out.append((m, encrypt_request(root, stacks[m], img, 1000 * seed + i)))
        return out

    # warm every slot (worker server) or every group size (batch server) on every resolution,
    # then the service time of each resolution alone
    for m in sizes:
        warm = [(m, encrypt_request(root, stacks[m], np.zeros((4, m, m)), 7))]
        if args.server == "batch":
            for b in server.sizes:
                server.serve([Request(i, 0.0, mm, co) for i, (mm, co) in enumerate(warm * b)])
        else:
            server.serve([Request(i, 0.0, mm, co) for i, (mm, co) in enumerate(warm * len(server.workers))])
    mem["after_warm_free_gb"] = torch.cuda.mem_get_info()[0] / 1e9
    alone = {}
    for m in sizes:
        co = encrypt_request(root, stacks[m], rng.uniform(0, 1, (4, m, m)), 9)
        ts = []
        for _ in range(3):
            r = server.serve([Request(0, 0.0, m, co)])[0]
            ts.append(r.finish - r.start)
        alone[m] = float(np.median(ts))
    mean_service = float(sum(alone[m] * p for m, p in zip(sizes, probs)))
    # capacity: closed-loop saturation throughput of the request mix (a burst all arriving at 0)
    burst = make(16 if args.server == "batch" else max(16, 4 * len(server.workers)), 3)
    done = server.serve([Request(i, 0.0, m, co) for i, (m, co) in enumerate(burst)])
    makespan = max(r.finish for r in done) - min(r.start for r in done)
    capacity = len(burst) / makespan
    reqs = make(args.requests, 1)
    results = []
    for frac in [float(x) for x in args.rates.split(",")]:
        rate = frac * capacity
        arr = workloads.poisson_arrivals(len(reqs), rate, seed=2)
        done = server.serve([Request(i, float(a), m, co) for i, ((m, co), a) in enumerate(zip(reqs, arr))])
        st = latency_stats(done)
        st.update({"load": frac, "arrival_rate_per_s": rate})
        results.append(st)
    line = {"workload": "serving: Poisson stream of %s images through 4 x [conv3x3+BN, deg-16 GELU, "
                        "avgpool], widths %s, 2N=2^16, 33+11 primes" % ("/".join(map(str, sizes)), widths),
            "conv": args.conv, "server": args.server,
            "workers": len(server.workers) if args.server == "workers" else None,
            "max_batch": args.max_batch if args.server == "batch" else None,
            "setup_s": setup_s, "key_bytes": H.he_key_bytes(root), "memory": mem,
            "service_ms_alone": {str(m): v * 1e3 for m, v in alone.items()},
            "capacity_images_per_s": capacity,
            "overlap_gain": capacity * mean_service,      # saturated throughput / one-at-a-time
            "runs": results}
    server.destroy()
    for s in stacks.values():
        s.destroy()
    H.he_ctx_destroy(root)
    return line


def main():
    """Serving benchmark: python -m paper_2306_09189_gb300.serve [--workers W] [--requests R]"""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--sizes", default="32,64")
    ap.add_argument("--rates", default="0.5,0.8,1.0", help="fractions of the measured capacity")
    ap.add_argument("--widths", default="4,16,32,64,64")
    ap.add_argument("--server", default="batch", choices=["batch", "workers"],
                    help="batch: stage-granularity continuous batching on one stream; workers: one "
                         "request per forked context and stream")
    ap.add_argument("--max-batch", type=int, default=4)
    ap.add_argument("--conv", default="diag", choices=["diag", "bsgs"],
                    help="convolution form: diagonal, or baby-step giant-step")
    args = ap.parse_args()
    line = run_benchmark(args)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
