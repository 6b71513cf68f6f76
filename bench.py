"""Benchmark: one CIFAR-shaped encrypted layer at ring 2^16 on one GB300.

Step = one pass of the whole hot path over one encrypted 16x32x32 image: hconv2d (3x3,
16->16, BN folded, 143 hoisted rotations, 144-term fused MAC, rescale, bias) followed by the
degree-16 Chebyshev GELU (15 relinearised products).  Parameters: n = 2^16, 20 ciphertext
primes (50 + 19 x 40 bits), 5 special primes, dnum 4, scale 2^40, input level 19.  Keys
(14.4 GB) and plaintexts (1.4 GB) are resident; every step streams them from HBM, so the
working set is far larger than L2 and no flush is needed.

Prints one JSON line (rank 0).  value = key switches per second (rotations + relins) over all
ranks; ms_per_step = layer latency.  The batched mode is the headline; the plain
per-ciphertext path is timed beside it, and the convolution alone (`conv_only`).  At N = 1 the
line also carries the batched ResNet block (`resnet_block`: 4 images at mixed levels, batched
vs plain), the ImageNet stem (`imagenet_stem`) and the serving loop (`serving`: Poisson
arrivals, p50/p99 latency and images/s), one full-ring bootstrap (`bootstrap`) and a whole
ResNet-20-shaped encrypted inference with bootstrapping (`resnet20`), each run on its own context
afterwards, and the oracle
on all host cores and on one (`cpu_baseline`).  N > 1 runs independent replicas
(the layer does not shard across GPUs).  --impl reference times the CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HE conv-layer ms and key-switches/s at 2N=2^16 on 1 GB300, batched vs plain"
WORKLOAD = "cifar layer: 16x32x32 conv3x3 16->16 + folded BN + degree-16 Chebyshev GELU, 2N=2^16, 20+5 primes"
LEVEL = 19
DEG = 16


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, ws):
    """The job's time: the max of a per-rank time over all ranks (NCCL on GPUs, gloo on CPU)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step_per_rank, ms_per_step, ws):
    """Whole-job throughput: the units every rank processed / the job's time (weak scaling)."""
    return ws * units_per_step_per_rank / (ms_per_step * 1e-3)


KERNEL_SRC = os.path.join(ROOT, "paper_2306_09189_gb300", "csrc", "kernels.cu")


def _traffic(profile, kernel):
    """DRAM bytes per launch of `kernel` from a committed ncu summary (lines 'key: value'),
    or None when the summary is missing, is for another kernel, or the kernel source changed
    since the counters were taken (its sha256 is recorded beside them)."""
    import hashlib
    try:
        kv = {}
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        with open(KERNEL_SRC) as f:
            src = f.read()
        b = src.index("// ==== fused key-switch + MAC kernels: begin")
        e = src.index("// ==== fused key-switch + MAC kernels: end")
        sha = hashlib.sha256(src[b:e].encode()).hexdigest()
        if kv.get("kernel_source_sha256") != sha or kernel not in kv.get("kernel", ""):
            return None
        return float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])
    except (OSError, KeyError, ValueError, IndexError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(sample_rotations=2):
    """The oracle as it stands on this host's cores: hoisted rotations of the layer input at
    the full ring (keys for them generated first, untimed)."""
    import workloads
    from oracle import layers as Ly
    from oracle.ckks import Context
    from oracle.params import C20
    o = Context(C20)
    wl = workloads.cifar_conv_bn(0)
    lin = Ly.image_layout(16, 32, o.N)
    ct = o.encrypt(Ly.pack(lin, wl.x)[0], LEVEL, nonce=1)
    amounts = [1, 32, 31, 33, 63, 64, 65, 95, 96, 97, 127, 128][:sample_rotations]
    amounts += [2 + i for i in range(max(0, sample_rotations - len(amounts)))]
    for a in amounts:
        o.gen_rotation_key(a)
    t0 = time.perf_counter()
    D = o.hoist(ct)
    for a in amounts:
        o.rotate_hoisted(ct, D, a)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": len(amounts) / dt, "unit": "key-switches/s", "cores": cores, "kind": "oracle",
            "sample": "%d hoisted rotations (ModUp once, inner product, ModDown) of the layer input "
                      "at n=2^16, level 19; %.1f s" % (len(amounts), dt)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_single_thread(sample_rotations=3):
    """The same oracle sample on one host core (OpenMP limited to one thread in a child process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", "import json, bench; print(json.dumps(bench.cpu_baseline(%d)))"
                        % sample_rotations], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode:
        return {"error": r.stderr.strip().splitlines()[-1:] or ["failed"]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        pass
    base = None
    for _ in range(args.steps):
        base = cpu_baseline(1)
        steps.append(1.0 / base["value"])
    ms = 1e3 * statistics.mean(steps)
    line = {"impl": "reference", "metric": METRIC, "value": 1e3 / ms, "unit": "key-switches/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "CPU oracle, one hoisted "
                                            "rotation of the layer input per step"},
            "cpu_baseline": {"value": 1e3 / ms, "unit": "key-switches/s", "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": 1e3 / ms, "unit": "key-switches/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BLOCK_LEVELS = (8, 12, 16, 19)
BLOCK_WORKLOAD = ("resnet basic block: 64x56x56 (64x64 frame, 8 shards of 8 channels), conv3x3+BN, "
                  "degree-16 Chebyshev GELU, conv3x3, residual; batch of 4 images at input levels "
                  "8/12/16/19, 2N=2^16, 20+5 primes")


def run_block(args, ws, rank, local, emit=True):
    """The batched form: one ResNet basic block over a batch of images at mixed levels.  Each
    conv of the batch is ONE fused-kernel launch over all images (groups of every image and
    level side by side); the GELU runs per ciphertext; the whole step is one CUDA graph."""
    import torch
    import workloads
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300 import host
    pr = host.cifar_params(seed=0)
    ctx = H.he_ctx_create(pr)
    H.he_ctx_set_option(ctx, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8, "twopass": H.HE_NTT_TWOPASS, "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED, "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[args.ntt])
    H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, {"auto": H.HE_KEY_STREAM_AUTO, "ldg": H.HE_KEY_STREAM_LDG,
                                                   "tma": H.HE_KEY_STREAM_TMA,
                                                   "split": H.HE_KEY_STREAM_SPLIT, "pk": H.HE_KEY_STREAM_PK,
                                                   "pk3": H.HE_KEY_STREAM_PK3, "pk1": H.HE_KEY_STREAM_PK1,
                                                   "pkt": H.HE_KEY_STREAM_PKT, "pk3l": H.HE_KEY_STREAM_PK3L,
                                                   "splitm": H.HE_KEY_STREAM_SPLITM}[args.key_stream])
    info = H.he_ctx_info(ctx)
    n, N = info["n"], info["slots"]
    q = info["q"]
    # --small: the profiling case (16 channels = 2 shards, two images at levels 8 and 12,
    # layer planned at level 12: a few GB on the device)
    levels = (8, 12) if args.small else BLOCK_LEVELS
    x0, (W1, b1), (W2, b2) = workloads.resnet_block(0, c=16 if args.small else 64)
    c, m = x0.shape[0], x0.shape[1]
    imgs = [x0] + [workloads.image(c, m, 10 + i) for i in range(len(levels) - 1)]
    top1 = max(levels)
    gdepth = host.ps_depth(DEG) if args.poly == "ps" else (DEG - 1).bit_length() + 1
    top2 = top1 - 1 - gdepth
    t_setup = time.perf_counter()
    lay = H.he_layout_image(c, m, N)
    if args.conv == "bsgs":
        def create(*a):
            return H.he_conv_create_bsgs(*a, args.bsgs_k)
    else:
        create = H.he_conv_create
    conv1 = create(ctx, lay, W1, b1, 1, 1, top1, pr.scale)
    lay1 = H.he_conv_out_layout(conv1)
    conv2 = create(ctx, lay1, W2, b2, 1, 1, top2, pr.scale)
    lay2 = H.he_conv_out_layout(conv2)
    H.he_keygen_rotations(ctx, sorted(set(H.he_conv_rotations(conv1)) | set(H.he_conv_rotations(conv2))))
    H.he_keygen_relin(ctx)
    cheb = host.chebyshev_coeffs("gelu", DEG, -8.0, 8.0)
    ns1, ns2 = lay.n_shards, lay1.n_shards
    xs = []
    for i, (img, lv) in enumerate(zip(imgs, levels)):
        xs += host.encrypt_image(ctx, lay, img, lv, pr.scale, nonce0=100 * i)
    y1 = [H.he_ct_alloc(ctx, top1 - 1) for _ in range(len(levels) * ns1)]
    y2 = [H.he_ct_alloc(ctx, top2 - 1) for _ in range(len(levels) * ns2)]
    # GELU output scale chosen so that conv2's output lands on the input's scale (residual)
    tgt = [pr.scale * float(q[lv - 1 - gdepth]) / float(q[top2]) for lv in levels]
    tgt_all = [t for t in tgt for _ in range(lay.n_shards)]
    setup_s = time.perf_counter() - t_setup

    products = host.ps_products(DEG) if args.poly == "ps" else DEG - 1
    ks_per_step = len(levels) * (H.he_conv_keyswitches(conv1) + H.he_conv_keyswitches(conv2) + ns1 * products)
    pt_bytes = sum(H.he_conv_n_terms(cv) * (lv + 1 + info["K"]) * n * 8 for cv, lv in ((conv1, top1), (conv2, top2)))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def step(mode):
        H.he_conv_run_batch(ctx, conv1, xs, y1, len(levels), mode, stream)
        one = H.he_poly_eval_ps if args.poly == "ps" else H.he_poly_eval
        many = H.he_poly_eval_ps_many if args.poly == "ps" else H.he_poly_eval_many
        if mode == H.HE_PLAIN:                   # the per-ciphertext path
            for i in range(len(levels)):
                for v in range(ns1):
                    one(ctx, y1[i * ns1 + v], cheb, tgt[i], stream)
        else:                                    # every ciphertext of a level through the products together
            many(ctx, y1, cheb, tgt_all, stream)
        H.he_conv_run_batch(ctx, conv2, y1, y2, len(levels), mode, stream)
        for i in range(len(levels)):
            for v in range(ns2):
                H.he_add(ctx, y2[i * ns2 + v], xs[i * ns1 + v], stream)

    step(H.HE_FUSED)
    torch.cuda.synchronize()
    H.he_graph_begin(ctx, stream)
    step(H.HE_FUSED)
    graph = H.he_graph_end(ctx, stream)

    def timed(mode, k, trace=None):
        for _ in range(args.warmup if mode == H.HE_FUSED else 1):
            if mode == H.HE_FUSED:
                H.he_graph_launch(graph, stream)
            else:
                step(mode)
        torch.cuda.synchronize()
        gk = None
        if trace:
            H.he_trace_start(trace)
        if mode == H.HE_FUSED:
            H.he_graph_begin(ctx, stream)
            for _ in range(k):
                step(mode)
            gk = H.he_graph_end(ctx, stream)
        l0 = H.he_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if gk is not None:
            H.he_graph_launch(gk, stream)
        else:
            for _ in range(k):
                step(mode)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), ws) / k
        launches = H.he_kernel_launches() - l0
        tr = H.he_trace_stop() if trace else None
        if gk is not None:
            H.he_graph_destroy(gk)
        return ms, launches, tr

    if args.profile_step:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step(H.HE_FUSED)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return
    # the roofline follows the kernel that carries the key switches of this step
    trace = args.trace
    if trace == "ipmac" and ("-> split" in H.he_ctx_tuning_log(ctx) or args.key_stream in ("split", "splitm")):
        trace = "rmac"
    clocks = Clocks(local)
    clocks.start()
    ms_f, launches_f, tr = timed(H.HE_FUSED, args.steps, trace)
    clk = clocks.stop()
    # sampled output check: image 0 (input level 8), decrypted, against the FP64 block with
    # the same polynomial
    from numpy.polynomial import chebyshev as C
    t1 = torch.nn.functional.conv2d(torch.tensor(imgs[0])[None], torch.tensor(W1), padding=1)[0].numpy() + b1[:, None, None]
    g1 = C.chebval(t1, cheb)
    want = torch.nn.functional.conv2d(torch.tensor(g1)[None], torch.tensor(W2), padding=1)[0].numpy() + b2[:, None, None] + imgs[0]
    got = host.decrypt_image(ctx, lay2, y2[:ns2])
    err = float(np.abs(got - want).max() / (want.max() - want.min()))
    ms_p, _, _ = timed(H.HE_PLAIN, 1)
    peaks, src = _peaks()
    roof = None
    if tr and tr["launches"]:
        per_launch_ms = tr["ms"] / tr["launches"]
        achieved = tr["bytes"] / tr["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": trace, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                "launches": tr["launches"], "ms_per_launch": per_launch_ms,
                "share_of_step": tr["ms"] / (ms_f * args.steps)}
    if rank == 0:
        line = {"metric": METRIC, "value": job_value(ks_per_step, ms_f, ws), "unit": "key-switches/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_f,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": BLOCK_WORKLOAD if not args.small else "profiling case: " + BLOCK_WORKLOAD.replace("64x56x56", "16x56x56"),
                           "input_levels": list(levels),
                           "key_switches_per_step": ks_per_step, "images": len(levels),
                           "mode": "each conv of the batch is one fused launch over all images and levels",
                           "conv": args.conv,
                           "bsgs_giant_blocks": [H.he_conv_bsgs_giant(conv1), H.he_conv_bsgs_giant(conv2)],
                           "conv_keyswitches_per_image": [H.he_conv_keyswitches(conv1), H.he_conv_keyswitches(conv2)],
                           "cuda_graph": True, "key_stream": args.key_stream,
                           "autotuner": H.he_ctx_tuning_log(ctx).strip().splitlines(),
                           "setup_s": setup_s,
                           "l2": "inputs larger than L2 (%.1f GB of keys, %.1f GB of plaintexts)"
                                 % (H.he_key_bytes(ctx) / 1e9, pt_bytes / 1e9),
                           "parallelism": "replicas" if ws > 1 else "single"},
                "plain": {"ms_per_step": ms_p, "value": ws * ks_per_step / (ms_p * 1e-3),
                          "batched_speedup": ms_p / ms_f,
                          "note": "image by image, per-ciphertext key switches, same plaintexts"
                                  + (" (per-rotation BSGS)" if args.conv == "bsgs" else "")},
                "check": {"image": 0, "input_level": levels[0], "max_err_rel_range": err,
                          "tolerance": 2.0 ** -20},
                "gpu_launches": int(launches_f), "roofline": roof, "clocks": clk}
        if emit:
            print(json.dumps(line), flush=True)
    H.he_ctx_check(ctx, stream)
    H.he_graph_destroy(graph)
    H.he_conv_destroy(conv1)
    H.he_conv_destroy(conv2)
    for ct in xs + y1 + y2:
        H.he_ct_free(ct)
    H.he_ctx_destroy(ctx)
    return line if rank == 0 else None


HEAD_WORKLOAD = ("resnet head: 64x8x8 feature map (one shard, 8 copies), pool-linear to 10 logits "
                 "(global average pool fused with the linear layer), batch of 8 images at level 4, "
                 "2N=2^16, 20+5 primes")


def run_head(args, ws, rank, local):
    """Pool-linear head of a ResNet (Sec. 4, Other Layers) over a batch of images: per image one
    weighted MAC per logit, log2 N rotate-and-add shifts (each one fused launch over the 10
    logits), the one-hot mask MAC; the batch step is one CUDA graph."""
    import torch
    import workloads
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300 import host
    pr = host.cifar_params(seed=0)
    ctx = H.he_ctx_create(pr)
    H.he_ctx_set_option(ctx, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8, "twopass": H.HE_NTT_TWOPASS, "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED, "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[args.ntt])
    N = H.he_ctx_info(ctx)["slots"]
    level, n_img = 4, 8
    x0, W, b = workloads.resnet_head(0)
    c, m = x0.shape[0], x0.shape[1]
    imgs = [x0] + [workloads.resnet_head(10 + i)[0] for i in range(n_img - 1)]
    lay = H.he_layout_image(c, m, N)
    L = H.he_pool_linear_create(ctx, lay, W, b, level, pr.scale)
    H.he_keygen_rotations(ctx, H.he_linear_rotations(L))
    xs = [host.encrypt_image(ctx, lay, img, level, pr.scale, nonce0=40 * i) for i, img in enumerate(imgs)]
    ys = [H.he_ct_alloc(ctx, level - 2) for _ in range(n_img)]
    ks_per_step = n_img * H.he_linear_keyswitches(L)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def step():
        for i in range(n_img):
            H.he_linear_run(ctx, L, xs[i], ys[i], stream)

    step()
    torch.cuda.synchronize()
    trace = args.trace
    if trace == "ipmac" and "-> split" in H.he_ctx_tuning_log(ctx):
        trace = "rmac"
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    H.he_trace_start(trace)
    H.he_graph_begin(ctx, stream)
    for _ in range(args.steps):
        step()
    gk = H.he_graph_end(ctx, stream)
    clocks = Clocks(local)
    clocks.start()
    l0 = H.he_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.he_graph_launch(gk, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = H.he_kernel_launches() - l0
    tr = H.he_trace_stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws) / args.steps
    H.he_graph_destroy(gk)
    got = H.he_decrypt(ctx, ys[0], N)[:W.shape[0]]
    want = W @ imgs[0].mean(axis=(1, 2)) + b
    err = float(np.abs(got - want).max() / (want.max() - want.min()))
    # the packed form of the same head (n' hoisted rotations, log2(N/n') shifts), timed the same way
    Lp = H.he_pool_linear_create_packed(ctx, lay, W, b, level, pr.scale)
    H.he_keygen_rotations(ctx, H.he_linear_rotations(Lp))
    for i in range(n_img):
        H.he_linear_run(ctx, Lp, xs[i], ys[i], stream)
    for _ in range(args.warmup):
        for i in range(n_img):
            H.he_linear_run(ctx, Lp, xs[i], ys[i], stream)
    torch.cuda.synchronize()
    H.he_graph_begin(ctx, stream)
    for _ in range(args.steps):
        for i in range(n_img):
            H.he_linear_run(ctx, Lp, xs[i], ys[i], stream)
    gp = H.he_graph_end(ctx, stream)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    H.he_graph_launch(gp, stream)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_pk = max_over_ranks(e2.elapsed_time(e3), ws) / args.steps
    H.he_graph_destroy(gp)
    got_pk = H.he_decrypt(ctx, ys[0], N)[:W.shape[0]]
    err_pk = float(np.abs(got_pk - want).max() / (want.max() - want.min()))
    ks_pk = H.he_linear_keyswitches(Lp)
    H.he_linear_destroy(Lp)
    peaks, src = _peaks()
    roof = None
    if tr and tr["launches"]:
        per_launch_ms = tr["ms"] / tr["launches"]
        achieved = tr["bytes"] / tr["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": trace, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                "launches": tr["launches"], "ms_per_launch": per_launch_ms,
                "share_of_step": tr["ms"] / (ms * args.steps)}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_value(ks_per_step, ms, ws), "unit": "key-switches/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": HEAD_WORKLOAD, "images": n_img, "input_level": level,
                       "key_switches_per_step": ks_per_step, "ms_per_image": ms / n_img, "cuda_graph": True,
                       "autotuner": H.he_ctx_tuning_log(ctx).strip().splitlines()[:3],
                       "l2": "working set below L2 (level 4: 10 partial sums of 5+5 limbs); keys %.2f GB"
                             % (H.he_key_bytes(ctx) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "check": {"image": 0, "max_err_rel_range": err, "tolerance": 2.0 ** -20},
            "packed": {"ms_per_step": ms_pk, "ms_per_image": ms_pk / n_img, "key_switches_per_image": ks_pk,
                       "speedup": ms / ms_pk, "check_max_err_rel_range": err_pk,
                       "note": "the same head in packed form: weights pre-rotated so one raised-basis stage of "
                               "n' = 16 hoisted rotations and log2(N/16) shifts give every logit its slot"},
            "gpu_launches": int(launches), "roofline": roof, "clocks": clk}), flush=True)
    H.he_ctx_check(ctx, stream)
    H.he_linear_destroy(L)
    for ct in [x for xi in xs for x in xi] + ys:
        H.he_ct_free(ct)
    H.he_ctx_destroy(ctx)


STEM_WORKLOAD = ("imagenet stem: 3x224x224 in channel shards (256 frame, 2 shards per channel), conv7x7/2 "
                 "3->64 pad 3 in the factored form (masks, then integer weights) with the stride-2 select, "
                 "-> 112x112x64 (32 shards) -> 2x2 avgpool -> 56x56x64 (8 shards); 2N=2^16, 20+5 primes")


BOOT_WORKLOAD = ("bootstrap: one level-0 ciphertext (2^15 real slots, scale 2^40) to level 8 of 23; "
                 "2N=2^16, 24+6 primes of 50 bits, weight-64 secret; ModRaise, 3 CoeffToSlot levels, "
                 "EvalMod (degree-59 Chebyshev cosine, 2 double angles), 3 SlotToCoeff levels")


def cpu_baseline_bootstrap():
    """The oracle on this host's cores for a bounded sample of the bootstrap at the full ring:
    ModRaise and the first CoeffToSlot level (32 diagonals, 16 rotations at level 23) of the B24
    chain, keys for it generated first (untimed)."""
    from oracle import bootstrap as OB
    from oracle.ckks import Context
    from oracle.params import B24
    o = Context(B24)
    plan = OB.BootPlan(o)
    for a in plan.cts[0].rotations():
        o.gen_rotation_key(a)
    z = np.random.default_rng(7).uniform(-1, 1, o.N)
    ct = o.encrypt(z, 0, 2.0 ** 40, nonce=1)
    pts = plan.plaintexts(o, "cts", 0)
    t0 = time.perf_counter()
    x = o.modraise(ct)
    x.scale = float(o.q[0]) * plan.cfg.K
    OB.lintrans_he(o, x, plan.cts[0], pts)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": dt, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": "ModRaise + the first CoeffToSlot level (32 diagonals, 16 hoisted rotations, "
                      "level 23) at n=2^16"}


def run_bootstrap(args, ws, rank, local, emit=True):
    """One bootstrap per step (the paper's largest cost, Sec. 5 tables), the whole pipeline
    captured as a CUDA graph; the decrypted output is compared with the input message."""
    import torch
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300 import host
    pr = host.bootstrap_params(seed=0)
    ctx = H.he_ctx_create(pr)
    H.he_ctx_set_option(ctx, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8,
                                            "twopass": H.HE_NTT_TWOPASS,
                                            "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED, "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[args.ntt])
    N = H.he_ctx_info(ctx)["slots"]
    t_setup = time.perf_counter()
    bt = H.he_boot_create(ctx)
    H.he_keygen_rotations(ctx, H.he_boot_rotations(bt))
    H.he_keygen_conjugation(ctx)
    H.he_keygen_relin(ctx)
    info = H.he_boot_info(bt)
    z = np.random.default_rng(7).uniform(-1, 1, N)
    x = H.he_ct_alloc(ctx, 0)
    H.he_encrypt(ctx, z, 0, 2.0 ** 40, 1, x)
    y = H.he_ct_alloc(ctx, info["out_level"])
    ts = torch.cuda.Stream()                              # graphs capture a created stream
    stream = ts.cuda_stream
    for _ in range(args.warmup):                          # first run: autotuner, buffers
        H.he_bootstrap(ctx, bt, x, y, stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    if args.profile_step:                                 # one eager bootstrap for a profiler
        torch.cuda.profiler.start()
        H.he_bootstrap(ctx, bt, x, y, stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        H.he_boot_destroy(bt)
        H.he_ctx_destroy(ctx)
        return None
    H.he_graph_begin(ctx, stream)
    H.he_bootstrap(ctx, bt, x, y, stream)
    graph = H.he_graph_end(ctx, stream)
    H.he_graph_launch(graph, stream)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(H.he_decrypt(ctx, y, N) - z)))
    # the timed region: K bootstraps in one graph, the fused key-switch kernel traced
    trace = args.trace
    H.he_trace_start(trace)
    H.he_graph_begin(ctx, stream)
    for _ in range(args.steps):
        H.he_bootstrap(ctx, bt, x, y, stream)
    gk = H.he_graph_end(ctx, stream)
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    torch.cuda.synchronize()
    l0 = H.he_kernel_launches()
    e0.record(ts)
    H.he_graph_launch(gk, stream)
    e1.record(ts)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (H.he_kernel_launches() - l0) / args.steps
    tr = H.he_trace_stop()
    peaks, src = _peaks()
    roof = None
    if tr and tr["launches"]:
        per = tr["ms"] / tr["launches"]
        ach = tr["bytes"] / tr["launches"] / (per * 1e-3) / 1e9
        roof = {"kernel": trace, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                "launches": tr["launches"] / args.steps, "ms_per_launch": per,
                "share_of_step": tr["ms"] / (ms * args.steps)}
    # eager (no graph) for comparison, and the oracle's sample beside it
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        H.he_bootstrap(ctx, bt, x, y, stream)
    torch.cuda.synchronize()
    eager_ms = (time.perf_counter() - t0) * 1e3 / 3
    # the bootstrap with its error bootstrapped once more and subtracted (MetaBTS, Appendix)
    ym = H.he_ct_alloc(ctx, info["out_level"])
    H.he_bootstrap_meta(ctx, bt, x, ym, 10, stream)
    torch.cuda.synchronize()
    H.he_graph_begin(ctx, stream)
    H.he_bootstrap_meta(ctx, bt, x, ym, 10, stream)
    gm = H.he_graph_end(ctx, stream)
    H.he_graph_launch(gm, stream)
    torch.cuda.synchronize()
    err_m = float(np.max(np.abs(H.he_decrypt(ctx, ym, N) - z)))
    km = max(1, args.steps // 2)
    e0.record(ts)
    for _ in range(km):
        H.he_graph_launch(gm, stream)
    e1.record(ts)
    torch.cuda.synchronize()
    meta = {"ms": e0.elapsed_time(e1) / km, "output_level": H.he_ct_level(ym), "max_abs_error": err_m,
            "bits": -float(np.log2(err_m)) if err_m > 0 else None, "kb": 10}
    H.he_graph_destroy(gm)
    H.he_ct_free(ym)
    line = {"metric": "bootstrap ms at 2N=2^16 on 1 GB300", "value": ms, "unit": "ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": BOOT_WORKLOAD, "key_switches_per_step": info["keyswitches"],
                       "input_levels": [0], "output_level": info["out_level"], "setup_s": setup_s,
                       "key_bytes": H.he_key_bytes(ctx), "cuda_graph": True},
            "eager_ms": eager_ms, "gpu_launches": int(round(launches)), "roofline": roof, "meta": meta,
            "check": {"max_abs_error": err, "bits": -float(np.log2(err)) if err > 0 else None},
            "clocks": ck}
    H.he_graph_destroy(graph)
    H.he_graph_destroy(gk)
    H.he_boot_destroy(bt)
    for c in (x, y):
        H.he_ct_free(c)
    H.he_ctx_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_bootstrap()
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    return line if rank == 0 else None


RESNET20_WORKLOAD = ("resnet-20 (CIFAR, 3x32x32): 3x3 stem, 3 stages x 3 basic blocks at 16/32/64 channels "
                     "(stride 2 and 1x1 shortcut at stages 2-3), folded BN, degree-16 GELU, pool-linear head; "
                     "bootstrapped wherever the levels run out; 2N=2^16, 24+6 primes of 50 bits")


def run_resnet20(args, ws, rank, local, emit=True):
    """One encrypted ResNet-20-shaped inference per step (the paper's Sec. 5 networks, whose CPU
    latencies it tabulates): the first image plans every layer and generates its keys, the next
    ones are timed; the logits are compared with the FP64 network with the same polynomial."""
    import torch
    import workloads
    from paper_2306_09189_gb300 import host
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300.network import EncryptedResNet
    net = workloads.resnet20(0)
    cheb = host.chebyshev_coeffs("gelu", workloads.GELU_DEGREE, -workloads.GELU_BOUND, workloads.GELU_BOUND)
    want = workloads.resnet20_forward(net, cheb)
    t0 = time.perf_counter()
    r = EncryptedResNet(host.bootstrap_params(0), net, cheb)
    r.infer(net["x"])                                      # plans, keys, autotuner
    setup_s = time.perf_counter() - t0
    steps = max(1, min(args.steps, 5))
    r.timing, r.counts = {}, {}
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    for i in range(steps):
        got = r.infer(net["x"], nonce0=100 * (i + 1))
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / steps
    ck = clocks.stop()
    err = float(np.max(np.abs(got - want)))
    line = {"metric": "encrypted ResNet-20 inference latency on 1 GB300", "value": sec, "unit": "s/image",
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": sec * 1e3, "higher_is_better": False,
            "dtype": "u64", "data": "synthetic weights and image",
            "config": {"workload": RESNET20_WORKLOAD, "setup_s": setup_s,
                       "key_bytes": H.he_key_bytes(r.ctx)},
            "breakdown_s": {k: v / steps for k, v in r.timing.items()},
            "counts": {k: v // steps for k, v in r.counts.items()},
            "check": {"max_abs_logit_error": err, "logit_range": float(np.max(want) - np.min(want))},
            "paper_context": "multiplexed ResNet-20, CIFAR-10: 486 s per image on a 32-core Threadripper 3970X "
                             "(OpenFHE, 2^14-slot shards, 59-bit scales)",
            "clocks": ck}
    r.close()
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    return line if rank == 0 else None


def run_stem(args, ws, rank, local, emit=True):
    """The ImageNet-shaped sharded stem (config 3): the factored channel-shard conv with stride 2
    (the select runs on 128 channel shards), then the 2x2 average pool; one CUDA graph per step.
    The per-rotation modes would hold every rotated shard of the select (hundreds of GB), so
    only the fused (raised-basis) form runs here."""
    import torch
    import workloads
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300 import host
    pr = host.cifar_params(seed=0)
    ctx = H.he_ctx_create(pr)
    H.he_ctx_set_option(ctx, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8, "twopass": H.HE_NTT_TWOPASS, "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED, "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[args.ntt])
    H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, {"auto": H.HE_KEY_STREAM_AUTO, "ldg": H.HE_KEY_STREAM_LDG,
                                                   "tma": H.HE_KEY_STREAM_TMA,
                                                   "split": H.HE_KEY_STREAM_SPLIT, "pk": H.HE_KEY_STREAM_PK,
                                                   "pk3": H.HE_KEY_STREAM_PK3, "pk1": H.HE_KEY_STREAM_PK1,
                                                   "pkt": H.HE_KEY_STREAM_PKT, "pk3l": H.HE_KEY_STREAM_PK3L,
                                                   "splitm": H.HE_KEY_STREAM_SPLITM}[args.key_stream])
    N = H.he_ctx_info(ctx)["slots"]
    wl = workloads.imagenet_stem(0)
    c, m = wl.x.shape[0], wl.x.shape[1]
    level = 19
    t_setup = time.perf_counter()
    lay = H.he_layout_image(c, m, N)
    conv = H.he_conv_create_factored(ctx, lay, wl.W, wl.bias, wl.stride, wl.pad, level, pr.scale)
    lay1 = H.he_conv_out_layout(conv)
    l1 = H.he_conv_out_level(conv)
    pool = H.he_pool_create(ctx, lay1, l1)
    lay2 = H.he_pool_out_layout(pool)
    H.he_keygen_rotations(ctx, sorted(set(H.he_conv_rotations(conv)) | set(H.he_pool_rotations(pool))))
    ks_per_step = H.he_conv_keyswitches(conv) + H.he_pool_keyswitches(pool)
    xs = host.encrypt_image(ctx, lay, wl.x, level, pr.scale, nonce0=1)
    y = [H.he_ct_alloc(ctx, l1) for _ in range(lay1.n_shards)]
    z = [H.he_ct_alloc(ctx, l1 - 2) for _ in range(lay2.n_shards)]
    setup_s = time.perf_counter() - t_setup
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def step():
        H.he_conv_run(ctx, conv, xs, y, H.HE_FUSED, stream)
        H.he_pool_run(ctx, pool, y, z, H.HE_FUSED, stream)

    step()
    torch.cuda.synchronize()
    if args.profile_step:
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return
    H.he_graph_begin(ctx, stream)
    step()
    graph = H.he_graph_end(ctx, stream)
    for _ in range(args.warmup):
        H.he_graph_launch(graph, stream)
    torch.cuda.synchronize()
    trace = args.trace                       # the pooling stages' fused launches dominate the stem
    H.he_trace_start(trace)
    H.he_graph_begin(ctx, stream)
    for _ in range(args.steps):
        step()
    gk = H.he_graph_end(ctx, stream)
    clocks = Clocks(local)
    clocks.start()
    l0 = H.he_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.he_graph_launch(gk, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), ws) / args.steps
    launches = H.he_kernel_launches() - l0
    tr = H.he_trace_stop()
    # sampled output check: output shards 0 and 1 (channels 0..15) against FP64
    want = torch.nn.functional.avg_pool2d(
        torch.nn.functional.conv2d(torch.tensor(wl.x)[None], torch.tensor(wl.W), stride=2, padding=3), 2)[0].numpy()
    chan, row0 = lay2.tables()
    got = np.stack([H.he_decrypt(ctx, z[u], N) for u in range(lay2.n_shards)])
    img = host.unpack(lay2, got)
    err = float(np.abs(img - want).max() / (want.max() - want.min()))
    peaks, src = _peaks()
    roof = None
    if tr and tr["launches"]:
        per = tr["ms"] / tr["launches"]
        ach = tr["bytes"] / tr["launches"] / (per * 1e-3) / 1e9
        roof = {"kernel": trace, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": src, "launches": tr["launches"],
                "ms_per_launch": per, "share_of_step": tr["ms"] / (ms * args.steps)}
    if rank == 0:
        line = {"metric": METRIC, "value": job_value(ks_per_step, ms, ws), "unit": "key-switches/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": STEM_WORKLOAD, "key_switches_per_step": ks_per_step,
                           "input_level": level, "output_level": l1 - 2, "cuda_graph": True,
                           "shards": [lay.n_shards, lay1.n_shards, lay2.n_shards],
                           "autotuner": H.he_ctx_tuning_log(ctx).strip().splitlines(), "setup_s": setup_s,
                           "l2": "inputs larger than L2 (%.1f GB of keys)" % (H.he_key_bytes(ctx) / 1e9),
                           "parallelism": "replicas" if ws > 1 else "single"},
                "plain": None, "plain_note": "per-rotation modes would hold every rotated shard of the 128-shard select",
                "check": {"max_err_rel_range": err, "tolerance": 2.0 ** -20},
                "gpu_launches": int(launches), "roofline": roof, "clocks": clk}
        if emit:
            print(json.dumps(line), flush=True)
    H.he_ctx_check(ctx, stream)
    H.he_graph_destroy(gk)
    H.he_graph_destroy(graph)
    H.he_conv_destroy(conv)
    H.he_pool_destroy(pool)
    for ct in xs + y + z:
        H.he_ct_free(ct)
    H.he_ctx_destroy(ctx)
    return line if rank == 0 else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--trace", default="ipmac", help="kernel whose launches the roofline uses")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ResNet-block, ImageNet-stem and serving figures the default line carries")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: same ring, 2-channel 32x32 conv (17 rotations, ~2 GB of keys)")
    ap.add_argument("--profile-step", action="store_true",
                    help="set up, warm up, then run one batched step between cudaProfilerStart/Stop")
    ap.add_argument("--key-stream", default="auto",
                    choices=["auto", "ldg", "tma", "split", "pk", "pk3", "pk1", "pkt", "pk3l", "splitm"],
                    help="key-switch + MAC form: autotuned (default), the fused kernel with vector "
                         "loads or a TMA tile pipeline, or the split form (inner products, then MAC)")
    ap.add_argument("--no-graph", action="store_true", help="launch the fused step eagerly, not as a CUDA graph")
    ap.add_argument("--conv", default="diag", choices=["diag", "bsgs"],
                    help="convolution form of the ResNet block: diagonal (one rotation per amount) or "
                         "baby-step giant-step")
    ap.add_argument("--bsgs-k", type=int, default=0,
                    help="giant stride (blocks) of the baby-step giant-step convolutions; 0 = cost model")
    ap.add_argument("--ntt", default="twopass", choices=["onepass", "onepass8", "twopass", "twopass-corrected", "twopass-shuffle"],
                    help="NTT at n = 2^16: one launch per limb on a 16-CTA cluster (onepass), on an "
                         "8-CTA cluster (onepass8), or the two-pass column/row form (its forward "
                         "butterflies without the per-butterfly correction when the primes allow, "
                         "or with it: twopass-corrected; twopass-shuffle: the row pass's transposes by "
                         "warp shuffles)")
    ap.add_argument("--poly", default="ps", choices=["ps", "tree"],
                    help="GELU evaluation: Paterson-Stockmeyer (default) or the binary tree")
    ap.add_argument("--workload", default="cifar-layer",
                    choices=["cifar-layer", "resnet-block", "imagenet-stem", "resnet-head", "bootstrap",
                             "resnet20"],
                    help="cifar-layer: the headline layer; resnet-block: the batched mixed-level block; "
                         "imagenet-stem: the channel-shard stem with stride 2 and average pool; "
                         "resnet-head: the pool-linear head; bootstrap: one full-ring bootstrap; "
                         "resnet20: a whole ResNet-20-shaped network with bootstrapping")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.workload in ("resnet-block", "imagenet-stem", "resnet-head", "bootstrap", "resnet20"):
        {"resnet-block": run_block, "imagenet-stem": run_stem, "resnet-head": run_head,
         "bootstrap": run_bootstrap, "resnet20": run_resnet20}[args.workload](args, ws, rank, local)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    import workloads
    from paper_2306_09189_gb300 import hegpu as H
    from paper_2306_09189_gb300 import host

    pr = host.cifar_params(seed=0)
    ctx = H.he_ctx_create(pr)
    H.he_ctx_set_option(ctx, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8, "twopass": H.HE_NTT_TWOPASS, "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED, "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[args.ntt])
    H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, {"auto": H.HE_KEY_STREAM_AUTO, "ldg": H.HE_KEY_STREAM_LDG,
                                                   "tma": H.HE_KEY_STREAM_TMA,
                                                   "split": H.HE_KEY_STREAM_SPLIT, "pk": H.HE_KEY_STREAM_PK,
                                                   "pk3": H.HE_KEY_STREAM_PK3, "pk1": H.HE_KEY_STREAM_PK1,
                                                   "pkt": H.HE_KEY_STREAM_PKT, "pk3l": H.HE_KEY_STREAM_PK3L,
                                                   "splitm": H.HE_KEY_STREAM_SPLITM}[args.key_stream])
    info = H.he_ctx_info(ctx)
    n, N = info["n"], info["slots"]
    wl = workloads.cifar_conv_bn(0, c=2) if args.small else workloads.cifar_conv_bn(0)
    lay = H.he_layout_image(wl.x.shape[0], 32, N)
    cheb = host.chebyshev_coeffs("gelu", DEG, -8.0, 8.0)
    x = host.encrypt_image(ctx, lay, wl.x, LEVEL, pr.scale, nonce0=1)[0]
    conv = H.he_conv_create(ctx, lay, wl.W, wl.bias, 1, 1, LEVEL, pr.scale)
    rots = H.he_conv_rotations(conv)
    H.he_keygen_rotations(ctx, rots)
    H.he_keygen_relin(ctx)
    # the same layer in baby-step giant-step form, timed beside the diagonal form
    conv_b = H.he_conv_create_bsgs(ctx, lay, wl.W, wl.bias, 1, 1, LEVEL, pr.scale, args.bsgs_k)
    H.he_keygen_rotations(ctx, H.he_conv_rotations(conv_b))
    y = H.he_ct_alloc(ctx, LEVEL - 1)
    products = host.ps_products(DEG) if args.poly == "ps" else DEG - 1
    ks_per_step = len(rots) + products
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()             # a created stream: the default one cannot be captured
    torch.cuda.set_stream(stream)

    poly = H.he_poly_eval_ps if args.poly == "ps" else H.he_poly_eval

    cur = {"conv": conv}

    def step(mode):
        H.he_conv_run(ctx, cur["conv"], [x], [y], mode, stream)
        poly(ctx, y, cheb, pr.scale, stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # the fused step as one CUDA graph (its first run builds, autotunes and allocates)
    step(H.HE_FUSED)
    torch.cuda.synchronize()
    H.he_graph_begin(ctx, stream)
    step(H.HE_FUSED)
    graph = H.he_graph_end(ctx, stream)

    def run(mode):
        if mode == H.HE_FUSED and not args.no_graph:
            H.he_graph_launch(graph, stream)
        else:
            step(mode)

    def timed(mode, k, trace=None):
        for _ in range(args.warmup):
            run(mode)
        barrier()
        graph_k = None
        if mode == H.HE_FUSED and not args.no_graph:
            # the K timed steps as one graph (captured while tracing: the traced kernel's
            # launches inside it carry their own event nodes)
            if trace:
                H.he_trace_start(trace)
            H.he_graph_begin(ctx, stream)
            for _ in range(k):
                step(mode)
            graph_k = H.he_graph_end(ctx, stream)
        elif trace:
            H.he_trace_start(trace)
        l0 = H.he_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if graph_k is not None:
            H.he_graph_launch(graph_k, stream)
        else:
            for _ in range(k):
                step(mode)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        launches = H.he_kernel_launches() - l0
        tr = H.he_trace_stop() if trace else None
        if graph_k is not None:
            H.he_graph_destroy(graph_k)
        ms = max_over_ranks(ms, ws)
        return ms / k, launches, tr

    if args.profile_step:
        for _ in range(args.warmup):
            run(H.HE_FUSED)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step(H.HE_FUSED)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return

    clocks = Clocks(local)
    clocks.start()
    ms_b, launches_b, tr = timed(H.HE_FUSED, args.steps, args.trace)
    clk = clocks.stop()
    ms_p, _, _ = timed(H.HE_PLAIN, max(1, args.steps // 2))
    ms_u, _, _ = timed(H.HE_BATCHED, max(1, args.steps // 2))
    # BSGS form: its first run builds and autotunes, then its own graph
    cur["conv"] = conv_b
    step(H.HE_FUSED)
    torch.cuda.synchronize()
    H.he_graph_destroy(graph)
    H.he_graph_begin(ctx, stream)
    step(H.HE_FUSED)
    graph = H.he_graph_end(ctx, stream)
    ms_bs, _, _ = timed(H.HE_FUSED, args.steps)
    ks_bsgs = H.he_conv_keyswitches(conv_b) + products
    cur["conv"] = conv


    # end to end through the C ABI with host buffers: pinned host ciphertext in, result out
    xin = H.he_ct_export_coeffs(ctx, x, n)
    h_in = torch.empty(xin.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64).reshape(xin.shape)
    h_in[:] = xin
    out_level = H.he_ct_level(y)                               # after the conv and the polynomial
    out_shape = (2, out_level + 1, n)
    h_out = torch.empty(int(np.prod(out_shape)), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    xe = H.he_ct_alloc(ctx, LEVEL)

    def e2e_body():
        H.he_conv_run(ctx, conv, [xe], [y], H.HE_FUSED, stream)
        poly(ctx, y, cheb, pr.scale, stream)

    H.he_ct_import_coeffs(xe, h_in, LEVEL, pr.scale, stream)
    e2e_body()
    torch.cuda.synchronize()
    H.he_graph_begin(ctx, stream)
    e2e_body()
    graph_e2e = H.he_graph_end(ctx, stream)

    def e2e_step():
        H.he_ct_import_coeffs(xe, h_in, LEVEL, pr.scale, stream)
        if args.no_graph:
            e2e_body()
        else:
            H.he_graph_launch(graph_e2e, stream)
        assert H.he_ct_level(y) == out_level
        H.load().he_ct_export_coeffs(y, H._p(h_out, H.U64P), H.stream_ptr(stream))

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    def conv_only_ms(cv, k):
        """The convolution alone (rotations, MAC, rescale, bias), K runs as one graph."""
        H.he_conv_run(ctx, cv, [x], [y], H.HE_FUSED, stream)
        barrier()
        H.he_graph_begin(ctx, stream)
        for _ in range(k):
            H.he_conv_run(ctx, cv, [x], [y], H.HE_FUSED, stream)
        g = H.he_graph_end(ctx, stream)
        for _ in range(args.warmup):
            H.he_graph_launch(g, stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.he_graph_launch(g, stream)
        e1.record(stream)
        barrier()
        H.he_graph_destroy(g)
        return max_over_ranks(e0.elapsed_time(e1), ws) / k

    conv_ms_bs = conv_only_ms(conv_b, args.steps)
    conv_ms = conv_only_ms(conv, args.steps)

    peaks, src = _peaks()
    roof = None
    if tr and tr["launches"]:
        per_launch_ms = tr["ms"] / tr["launches"]
        achieved = tr["bytes"] / tr["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": args.trace, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": _traffic("fused_kernel_cifar_layer_traffic.txt", args.trace),
                "algorithmic_bytes_per_launch": tr["bytes"] / tr["launches"],
                "peak_source": src, "launches": tr["launches"], "ms_per_launch": per_launch_ms,
                "share_of_step": tr["ms"] / (ms_b * args.steps)}
    mm_rate = H.he_bench_modmul(ctx, 152 * 8, 2048)
    mac_rate = H.he_bench_mac(ctx, 152 * 8, 4096)
    if roof is not None and tr.get("mulmods"):
        # integer pipe: the library counts the kernel's 64x64->128-bit multiply-accumulates; the
        # peak is the measured throughput of that operation with 8 independent chains per thread
        mm = tr["mulmods"] / tr["launches"] / (roof["ms_per_launch"] * 1e-3)
        roof["int"] = {"unit": "64x64->128-bit multiply-accumulates/s", "achieved": mm, "peak": mac_rate,
                       "frac": mm / mac_rate,
                       "peak_source": "he_bench_mac: 8 independent chains per thread, 152 x 8 blocks of 256 "
                                      "threads (measured on this GPU in this run)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": job_value(ks_per_step, ms_b, ws), "unit": "key-switches/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": "batched+fused: every rotation key streamed once "
                                                      "into a raised-basis MAC, one ModDown per output; "
                                                      "relinearised products of one operand level "
                                                      "batched",
                       "key_switches_per_step": ks_per_step, "key_stream": args.key_stream,
                       "ntt": args.ntt, "cuda_graph": not args.no_graph,
                       "autotuner": H.he_ctx_tuning_log(ctx).strip().splitlines(),
                       "rotations": int(len(rots)), "relins": products, "input_level": LEVEL,
                       "gelu": "degree-16 Chebyshev, %s" % ("Paterson-Stockmeyer" if args.poly == "ps" else "binary tree"),
                       "l2": "inputs larger than L2 (rotation keys %.1f GB streamed every step)" % (H.he_key_bytes(ctx) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "plain": {"ms_per_step": ms_p, "value": ws * ks_per_step / (ms_p * 1e-3),
                      "batched_speedup": ms_p / ms_b,
                      "note": "per-ciphertext launches, one ModDown per rotation"},
            "bsgs": {"ms_per_step": ms_bs, "key_switches_per_step": ks_bsgs,
                     "giant_blocks": H.he_conv_bsgs_giant(conv_b),
                     "speedup_vs_diagonal": ms_b / ms_bs, "speedup_vs_plain": ms_p / ms_bs,
                     "note": "same layer, baby-step giant-step convolution (tap shifts per input shard, "
                             "channel offsets per partial sum), both steps raised-basis fused stages"},
            "batched_unfused": {"ms_per_step": ms_u, "value": ws * ks_per_step / (ms_u * 1e-3),
                                "note": "all rotations per launch, one ModDown per rotation (bits equal plain)"},
            "e2e": {"value": ws * ks_per_step / (e2e_ms * 1e-3), "unit": "key-switches/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h_in.nbytes),
                    "d2h_bytes_per_step": int(np.prod(out_shape) * 8)},
            "gpu_launches": int(launches_b),
            "roofline": roof,
            "modmul_microbench_per_s": mm_rate,
            "mac_microbench_per_s": mac_rate,
            "clocks": clk,
            "conv_only": {"ms": conv_ms, "bsgs_ms": conv_ms_bs,
                          "gelu_ms": ms_b - conv_ms, "key_switches": int(len(rots)),
                          "note": "the convolution alone (hoisted rotations, fused MAC, one ModDown, "
                                  "rescale, bias), as one graph of K runs; gelu_ms = step - conv"},
        }
    H.he_ctx_check(ctx, stream)
    H.he_graph_destroy(graph)
    H.he_graph_destroy(graph_e2e)
    H.he_conv_destroy(conv)
    H.he_conv_destroy(conv_b)
    for c in (x, y, xe):
        H.he_ct_free(c)
    H.he_ctx_destroy(ctx)
    if ws == 1 and not args.no_extra:
        # the batched ResNet block (the survey's headline for batched vs plain) and the ImageNet
        # stem, each on its own context after the layer's is released
        for key, fn, k in (("resnet_block", run_block, 5), ("imagenet_stem", run_stem, 3),
                           ("bootstrap", run_bootstrap, 20), ("resnet20", run_resnet20, 3)):
            sub = argparse.Namespace(**vars(args))
            sub.steps, sub.warmup, sub.trace, sub.small, sub.profile_step = k, 3, "ipmac", False, False
            line[key] = _extra_summary(fn(sub, ws, rank, local, emit=False))
        # serving: Poisson streams of 32x32 and 64x64 requests (64 per load of 0.5, 0.8 and 1.0 of the
        # measured capacity) through the 4-layer stack at
        # 33 + 11 primes, continuous batching at stage granularity (p50/p99 and images/s)
        from paper_2306_09189_gb300 import serve
        sv = serve.run_benchmark(argparse.Namespace(sizes="32,64", widths="4,16,32,64,64", rates="0.5,0.8,1.0",
                                                    requests=64, conv="bsgs", server="batch", workers=4,
                                                    max_batch=4))
        line["serving"] = {k: sv[k] for k in ("workload", "server", "max_batch", "conv", "setup_s",
                                              "service_ms_alone", "capacity_images_per_s", "runs", "memory")}
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:              # the oracle baseline: rank 0 at N = 1 only
            line["cpu_baseline"] = cpu_baseline(48)          # ~10 s of oracle work on every core
            line["cpu_baseline"]["cpu_model"] = cpu_model()
            line["cpu_baseline"]["single_thread"] = cpu_baseline_single_thread(3)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _extra_summary(d):
    """The figures of a secondary workload's line that the headline line carries."""
    if d is None:
        return None
    keep = ("ms_per_step", "value", "unit", "steps", "plain", "check", "roofline", "clocks", "gpu_launches",
            "eager_ms", "cpu_baseline", "meta", "breakdown_s", "counts", "paper_context")
    out = {k: d[k] for k in keep if k in d}
    out["workload"] = d["config"]["workload"]
    for k in ("key_switches_per_step", "input_levels", "output_level", "setup_s", "l2",
              "conv_keyswitches_per_image", "shards"):
        if k in d["config"]:
            out[k] = d["config"][k]
    return out


if __name__ == "__main__":
    main()
