"""Benchmark of the GB300 RNS-CKKS hot path (PrivFT, arXiv 1908.06972).

Workload (one step): a batch of 64 ciphertexts at N = 2^16 on a 30-prime chain
(q_0: 60 bits, q_1..q_29: 50 bits; 4 special primes of 60 bits; digits of 4 primes),
levels drawn uniformly from 5..30, each put through HMUL + relinearisation followed by
a chain of 16 power-of-two rotations (steps 2^0 .. 2^14 and -1).  The batched path
issues each stage once for the whole batch (every key read once per launch, whatever the
levels); the plain path issues every op for every ciphertext separately.

Output: one JSON line (rank 0).  `value` is HE mult+relin per second of the batched
path with inputs resident in HBM (each counted mult+relin carries its 16 rotations);
`e2e` measures the same through the C ABI from page-locked host buffers: every step's
128 input ciphertexts are copied in (pft_ct_import_batch) and its 64 results copied out
(pft_ct_export_batch_async) inside the timed region, on an import and an export stream that
overlap the previous and next steps' compute (split.link_gbs: the host link's copy rates).  Further legs: the step as one CUDA-graph launch, the
plain path, encrypted fastText inference, the encrypted training step and the request
server.  `--impl reference` times the CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

LOGN, L, K_SP, ALPHA = 16, 30, 4, 4
FIRST, MID, SPECIAL = 60, 50, 60
SCALE = 2.0 ** 50
BATCH = 64
STEPS_ROT = [1 << i for i in range(15)] + [-1]
SEED = (0x5EED0001, 0x5EED0002, 0x5EED0003, 0x5EED0004)
WORKLOAD = ("N=2^16, 30 limbs (60 + 29x50 bits) + 4 special (60 bits), digits of 4 primes; "
            "batch 64 ciphertexts at levels U{5..30}; per ciphertext mul_relin then 16 chained "
            "rotations (2^0..2^14, -1)")
# Nominal integer figures (context only; the reported bound uses the measured multiply rates):
# 152 SMs x 64 32-bit IMAD per SM per clock x 2.07 GHz, 9 IMAD per Shoup butterfly.
SMS, IMAD_PER_CLK, SM_MHZ_MAX, IMAD_PER_MULMOD = 152, 64, 2070.0, 9
# DRAM bytes (read + written) per limb and pass of the N = 2^16 transform kernels: ncu
# dram__bytes_read.sum + dram__bytes_write.sum over the four two-pass launches of the
# 16 x 30-limb case (bench.py --case ntt), divided by their 4 x 480 limb-passes (the kernels
# with the reverse-order second pass and the evict-last row twiddles: 1913.7 MB; 1943.1 MB
# before those changes).
NTT_DRAM_BYTES_PER_LIMB_PASS = 0.9967e6


def alu_bound(lo, hi):
    """Butterflies/s the integer multiply pipe allows: each butterfly (a Shoup product with the
    estimated quotient) issues 5 multiplies that produce a high word and 4 low-word ones."""
    return 1.0 / (5.0 / hi + 4.0 / lo)


def levels():
    from paper_1908_06972_gb300 import synth
    return synth.batch_levels(BATCH, 5, 30)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x, device):
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, max_seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time.
    Ranks work on independent batches (weak scaling, no data-path collective)."""
    return units_per_rank * world / max_seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- GPU arm ------------------------------------------------------------------------------------
def run_gpu(args):
    import torch

    import paper_1908_06972_gb300 as pft
    from paper_1908_06972_gb300 import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pft.build()
    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, FIRST, MID, SPECIAL, SCALE, SEED,
                             flags=pft.PFT_COMPRESSED_KEYS if args.compressed_keys else 0)
    tune_report = None
    if AUTOTUNE[0]:
        pft.pft_autotune(ctx)
        tune_report = pft.pft_autotune_report(ctx)
    bfly_ceiling = pft.pft_bfly_ceiling(ctx) / 1e9  # G butterflies/s of the butterfly on register data
    mul_lo, mul_hi, mul_wide = pft.pft_mul_rates(ctx)  # measured 32-bit multiply issue rates
    pft.pft_keygen(ctx, STEPS_ROT, True)
    lv = levels()
    n = 1 << LOGN
    A, B = [], []
    for i, l in enumerate(lv):
        pa = pft.pft_encode(ctx, synth.slots(1000 + i + 7919 * rank, 256), SCALE, l)
        pb = pft.pft_encode(ctx, synth.slots(5000 + i + 7919 * rank, 256), SCALE, l)
        A.append(pft.pft_encrypt(ctx, pa, pft.PFT_ENC_SK, 2 * i))
        B.append(pft.pft_encrypt(ctx, pb, pft.PFT_ENC_SK, 2 * i + 1))
        pft.pft_pt_destroy(pa)
        pft.pft_pt_destroy(pb)
    C = [pft.pft_ct_create(ctx) for _ in range(BATCH)]

    def step_batched(a, b, c):
        pft.pft_mul_relin_batch(ctx, a, b, c)
        for s in STEPS_ROT:
            pft.pft_rotate_batch(ctx, c, s, c)

    def step_plain(a, b, c):
        for i in range(BATCH):
            pft.pft_mul_relin(ctx, a[i], b[i], c[i])
            for s in STEPS_ROT:
                pft.pft_rotate(ctx, c[i], s, c[i])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        barrier()
        return reduce_max(e0.elapsed_time(e1), "cuda")

    for _ in range(args.warmup):
        step_batched(A, B, C)
    # host cost of issuing one step into an idle queue (no back-pressure from the device): the
    # rate the host could sustain if the device were infinitely fast
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    step_batched(A, B, C)
    host_issue_ms = 1e3 * (time.perf_counter() - h0)
    torch.cuda.synchronize()
    # timed region: batched path, dominant kernel family timed with events on the library stream
    pft.pft_prof_start(args.roofline_kernel)
    with ClockSampler(local) as clk:
        ms = timed(lambda: step_batched(A, B, C), args.steps)
    k_ms, k_launches, all_launches, k_work = pft.pft_prof_stop()
    ms_step = ms / args.steps
    value = throughput(BATCH * args.steps, world, ms / 1e3)

    # the same step captured once as a CUDA graph and replayed (separate context: graph capture
    # needs the stream-ordered default allocator and a non-default stream)
    graph_value = graph_ctx_eager_value = None
    if args.graph:
        graph_value, graph_ctx_eager_value = graph_measure(pft, torch, synth, args.steps, args.warmup, rank, world)

    # plain one-op-per-launch path (same GPU, same inputs)
    plain = None
    if args.plain_steps > 0:
        step_plain(A, B, C)
        pm = timed(lambda: step_plain(A, B, C), args.plain_steps)
        plain = throughput(BATCH * args.plain_steps, world, pm / 1e3)

    # end to end through the C ABI from pinned host buffers
    host_in = []
    for i in range(BATCH):
        for h in (A[i], B[i]):
            arr = torch.empty((2, lv[i], n), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
            pft.pft_ct_export(ctx, h, arr)
            host_in.append((arr, pft.pft_ct_scale(h)))
    host_out = [torch.empty((2, l - 0, n), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64) for l in lv]
    h2d = sum(a.nbytes for a, _ in host_in)
    d2h = sum(o.nbytes for o in host_out)

    # Pipelined through the public API on two copy streams: step i+1's inputs are copied into one
    # of two fixed sets of input handles (pft_ct_import_batch_into, on the import stream) and step
    # i's results out of one of two sets of outputs into page-locked buffers
    # (pft_ct_export_batch_async, on the export stream) while the compute stream runs, so the two
    # directions use their own copy engines at the same time.  Events order the streams: an import
    # waits for the end of the step that last read its set, an export for the end of its step, a
    # step for its import and for the export that last read its outputs; the host never blocks
    # before the end, and every step's results are in host memory before the timed region ends.
    S = torch.cuda.current_stream()
    Ci, Ce = torch.cuda.Stream(), torch.cuda.Stream()
    C2 = [C, [pft.pft_ct_create(ctx) for _ in range(BATCH)]]
    IN2 = [[pft.pft_ct_create(ctx) for _ in range(2 * BATCH)] for _ in range(2)]
    outs2 = [host_out, [torch.empty(o.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
                        for o in host_out]]
    marks = []
    step_end = {}  # step -> event at the end of its compute

    def on_stream(strm, fn):
        pft.pft_set_stream(ctx, strm.cuda_stream)
        fn()
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(strm)
        pft.pft_set_stream(ctx, S.cuda_stream)
        return ev

    def import_into(k):
        if k - 2 in step_end:  # step k - 2 read this set of input handles
            Ci.wait_event(step_end.pop(k - 2))
        return on_stream(Ci, lambda: pft.pft_ct_import_batch_into(ctx, [arr for arr, _ in host_in],
                                                                  [sc for _, sc in host_in], IN2[k % 2]))

    host = {"import": 0.0, "compute": 0.0, "export": 0.0, "wait": 0.0}
    exported = {}

    def step_e2e(k, ready, last):
        h0 = time.perf_counter()
        nxt = import_into(k + 1) if not last else None
        h1 = time.perf_counter()
        S.wait_event(ready)
        if k - 2 in exported:
            S.wait_event(exported.pop(k - 2))  # the outputs of step k - 2 have been read
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(S)
        ins = IN2[k % 2]
        step_batched(ins[0::2], ins[1::2], C2[k % 2])
        ev[1].record(S)
        step_end[k] = ev[1]
        h2 = time.perf_counter()
        Ce.wait_event(ev[1])
        exported[k] = on_stream(Ce, lambda: pft.pft_ct_export_batch_async(ctx, C2[k % 2], outs2[k % 2]))
        h3 = time.perf_counter()
        for key, dt in (("import", h1 - h0), ("compute", h2 - h1), ("export", h3 - h2)):
            host[key] += dt
        marks.append(ev)
        return nxt

    def drain():
        h = time.perf_counter()
        Ci.synchronize()
        Ce.synchronize()
        S.synchronize()
        exported.clear()
        step_end.clear()
        host["wait"] += time.perf_counter() - h

    # warm-up over both sets, so that no buffer is allocated inside the timed region
    step_e2e(1, step_e2e(0, import_into(0), False), True)
    drain()
    barrier()
    marks.clear()
    for key in host:
        host[key] = 0.0
    t0 = time.perf_counter()
    ready = import_into(0)
    for k in range(args.steps):
        ready = step_e2e(k, ready, k == args.steps - 1)
    drain()
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, "cuda")
    e2e = throughput(BATCH * args.steps, world, e2e_s)
    e2e_split = {"compute_ms": round(sum(ev[0].elapsed_time(ev[1]) for ev in marks) / len(marks), 2),
                 "wall_ms": round(1e3 * e2e_s / args.steps, 2),
                 "host_ms": {key: round(1e3 * v / args.steps, 2) for key, v in host.items()},
                 "link_gbs": link_rates(host_in[0][0], host_out[0]),
                 "host_issue_ms_idle_queue": round(host_issue_ms, 2)}
    for h in C2[1] + IN2[0] + IN2[1]:
        pft.pft_ct_destroy(h)

    # roofline of the timed kernel family
    roof = None
    clk_med = clk.summary().get("sm_mhz")  # median SM clock sampled during the timed region
    if k_ms > 0 and args.roofline_kernel.startswith("ntt"):
        achieved = k_work / (k_ms / 1e3) / 1e9  # Gbutterfly/s (one Shoup mulmod each)
        peak = alu_bound(mul_lo, min(mul_hi, mul_wide)) / 1e9
        limb_passes = k_work / max(1, k_launches) / ((1 << LOGN) // 2 * 8)
        roof = {"bound": "alu", "kernel": args.roofline_kernel, "achieved": round(achieved, 2),
                "peak": round(peak, 2), "unit": "Gmulmod/s", "frac": round(achieved / peak, 4),
                "traffic": round(NTT_DRAM_BYTES_PER_LIMB_PASS * limb_passes),
                "algorithmic_bytes": round(limb_passes * (1 << LOGN) * 16),
                "traffic_source": "ncu DRAM bytes per limb-pass of the 16 x 30-limb transform case, "
                                  "times the mean limb-passes per launch in the step",
                "launches": k_launches, "kernel_ms": round(k_ms, 3),
                "kernel_share_of_step": round(k_ms / ms, 4),
                "peak_source": "derived from the multiply issue rates measured live (pft_mul_rates): "
                               "1 / (5 / high-word rate + 4 / low-word rate) butterflies/s; a butterfly is "
                               "5 multiplies producing a high word and 4 low-word multiply-adds",
                "mul_rates_per_sm_clk": {"lo": round(mul_lo / SMS / (SM_MHZ_MAX * 1e6), 1),
                                         "hi": round(mul_hi / SMS / (SM_MHZ_MAX * 1e6), 1),
                                         "wide": round(mul_wide / SMS / (SM_MHZ_MAX * 1e6), 1)},
                "peak_nominal_64imad": round(SMS * IMAD_PER_CLK * SM_MHZ_MAX * 1e6 / IMAD_PER_MULMOD / 1e9, 1),
                "arith_ceiling": round(bfly_ceiling, 1), "frac_of_arith_ceiling": round(achieved / bfly_ceiling, 4),
                "peak_at_median_clock": round(peak * clk_med / SM_MHZ_MAX, 2) if clk_med else None,
                "frac_at_median_clock": round(achieved / (peak * clk_med / SM_MHZ_MAX), 4) if clk_med else None,
                "arith_ceiling_source": "measured live: the transforms' butterfly on register data, no memory "
                                        "traffic (pft_bfly_ceiling)"}
    elif k_ms > 0:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
        achieved = k_work / (k_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": args.roofline_kernel, "achieved": round(achieved, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": None, "launches": k_launches, "kernel_ms": round(k_ms, 3),
                "kernel_share_of_step": round(k_ms / ms, 4)}

    ft = None
    if args.fasttext:
        ft = fasttext_measure(pft, torch, max(1, args.steps // 2), 1)
        if args.fasttext_l30:
            ft["level30"] = fasttext_measure_l30(pft, torch)
            ft["level30"]["frac_of_alu_bound"] = round(
                ft["level30"]["batched_gmulmod_s"] / (alu_bound(mul_lo, min(mul_hi, mul_wide)) / 1e9), 4)

    tr = None
    if args.train > 0:
        tr = train_measure(pft, torch, args.train, args.train_plain_docs, args.train_diag > 0)

    ops = None
    if args.ops > 0:
        ops = ops_measure(pft, torch, synth, ctx, args.ops)

    qu = None
    if args.queue > 0:
        qu = queue_measure(pft, torch, args.queue)
        qu["two_ring_keyswitch"] = rings_measure(pft, torch, synth, 10)

    sv = None
    if args.serve > 0:
        sv = serve_measure(pft, torch, args.serve, args.serve_rate, args.serve_budget_gib, args.serve_near,
                           args.serve_fig3 > 0)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_level)

    out = {"metric": "HE mult+relin/s at N=2^16; enc. fastText inferences/s, batched vs plain",
           "value": round(value, 3), "unit": "mult+relin/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "batch": BATCH, "levels_mean": round(float(np.mean(lv)), 2),
                      "l2": "inputs larger than L2 (%.1f GB of ciphertexts)" % (h2d / 1e9),
                      "parallelism": "replicas" if world > 1 else "single"},
           "plain_value": round(plain, 3) if plain else None,
           "graph_value": round(graph_value, 3) if graph_value else None,
           "graph_context_eager_value": round(graph_ctx_eager_value, 3) if graph_ctx_eager_value else None,
           "e2e": {"value": round(e2e, 3), "unit": "mult+relin/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "split": e2e_split},
           "gpu_launches": int(all_launches), "roofline": roof,
           "autotune": tune_report, "cpu_baseline": cpu, "clocks": clk.summary(),
           "fasttext": ft, "serving": sv, "training": tr, "job_queue": qu, "ops": ops}
    if rank == 0:
        print(json.dumps(out))
    for h in A + B + C:
        pft.pft_ct_destroy(h)
    pft.pft_ctx_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def graph_measure(pft, torch, synth, steps, warmup, rank, world):
    stream = torch.cuda.Stream()
    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, FIRST, MID, SPECIAL, SCALE, SEED, allocator=None,
                             stream=stream.cuda_stream)
    tune(pft, ctx)  # the transform plans of the main context's step (chosen per launch size)
    pft.pft_keygen(ctx, STEPS_ROT, True)
    A, B = [], []
    for i, l in enumerate(levels()):
        pa = pft.pft_encode(ctx, synth.slots(1000 + i + 7919 * rank, 256), SCALE, l)
        pb = pft.pft_encode(ctx, synth.slots(5000 + i + 7919 * rank, 256), SCALE, l)
        A.append(pft.pft_encrypt(ctx, pa, pft.PFT_ENC_SK, 2 * i))
        B.append(pft.pft_encrypt(ctx, pb, pft.PFT_ENC_SK, 2 * i + 1))
        pft.pft_pt_destroy(pa)
        pft.pft_pt_destroy(pb)
    C = [pft.pft_ct_create(ctx) for _ in range(BATCH)]

    def step():
        pft.pft_mul_relin_batch(ctx, A, B, C)
        for s in STEPS_ROT:
            pft.pft_rotate_batch(ctx, C, s, C)

    def timed(fn):
        stream.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return reduce_max(e0.elapsed_time(e1), "cuda")

    for _ in range(warmup):
        step()
    eager_ms = timed(step)  # the same context's eager step (stream-ordered allocator, no autotuning)
    pft.pft_graph_begin(ctx)
    step()
    g = pft.pft_graph_end(ctx)
    for _ in range(warmup):
        pft.pft_graph_launch(ctx, g)
    ms = timed(lambda: pft.pft_graph_launch(ctx, g))
    pft.pft_graph_destroy(g)
    for h in A + B + C:
        pft.pft_ct_destroy(h)
    pft.pft_ctx_destroy(ctx)
    return throughput(BATCH * steps, world, ms / 1e3), throughput(BATCH * steps, world, eager_ms / 1e3)


RG_WORKLOAD = ("key switching of the two serving rings in one step: N=2^16 (60 + 29x40 bits + 4 special, digits of "
               "4) and N=2^15 (60 + 17x40 bits + 2 special, digits of 2), 32 ciphertext pairs each at levels "
               "U{12..30} / U{12..18}, one batched HMUL + relinearisation per ring")


def rings_measure(pft, torch, synth, reps):
    """The key-switch stages of both serving rings (uneven ring sizes and levels) issued three
    ways: on one stream one ring after the other; on two streams concurrently; and captured
    together into one CUDA graph (the second stream forked from and joined back into the first)
    replayed as a single launch."""
    streams, ctxs, work = [], [], []
    for logn, lim, ksp, alpha, (lo, hi) in SV_RINGS:
        st = torch.cuda.Stream()
        ctx = pft.pft_ctx_create(logn, lim, ksp, alpha, 60, 40, 60, 2.0 ** 40, SEED, allocator=None,
                                 stream=st.cuda_stream)
        tune(pft, ctx)
        pft.pft_keygen(ctx, [], True)
        lv = synth.batch_levels(32, lo, hi, seed=logn)
        A, B = [], []
        for i, l in enumerate(lv):
            for lst, base in ((A, 100), (B, 300)):
                pt = pft.pft_encode(ctx, synth.slots(base + i, 64), 2.0 ** 40, l)
                lst.append(pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, base + i))
                pft.pft_pt_destroy(pt)
        C = [pft.pft_ct_create(ctx) for _ in lv]
        streams.append(st)
        ctxs.append(ctx)
        work.append((A, B, C))

    def both():
        for i in range(2):
            pft.pft_mul_relin_batch(ctxs[i], *work[i])

    def timed(fn, fork):
        """Events on stream 0; with fork the second stream starts after and ends before them."""
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        if fork:
            streams[1].wait_event(e0)
        for _ in range(reps):
            fn()
        if fork:
            j = torch.cuda.Event()
            j.record(streams[1])
            streams[0].wait_event(j)
        e1.record(streams[0])
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    both()
    out = {"workload": RG_WORKLOAD, "unit": "ms per step (both rings)"}
    pft.pft_set_stream(ctxs[1], streams[0].cuda_stream)  # one stream
    both()
    out["one_stream"] = round(timed(both, False), 3)
    pft.pft_set_stream(ctxs[1], streams[1].cuda_stream)  # each ring on its own stream
    out["two_streams"] = round(timed(both, True), 3)
    # one graph: capture on stream 0, fork stream 1 into the capture, join it back
    pft.pft_graph_begin(ctxs[0])
    f = torch.cuda.Event()
    f.record(streams[0])
    streams[1].wait_event(f)
    both()
    j = torch.cuda.Event()
    j.record(streams[1])
    streams[0].wait_event(j)
    g = pft.pft_graph_end(ctxs[0])
    pft.pft_graph_launch(ctxs[0], g)
    out["one_graph_launch"] = round(timed(lambda: pft.pft_graph_launch(ctxs[0], g), False), 3)
    pft.pft_graph_destroy(g)
    for ctx, (A, B, C) in zip(ctxs, work):
        for h in A + B + C:
            pft.pft_ct_destroy(h)
        pft.pft_ctx_destroy(ctx)
    return out


# ---- encrypted fastText inference (Sec. 3.1, Fig. 3) ------------------------------------------------
FT_M, FT_N, FT_C, FT_LEVEL, FT_BATCH = 32768, 64, 14, 3, 32
FT_WORKLOAD = ("vocab 32768, dim 64, 14 classes, weights N(0, 0.1^2); Zipf(1.1) documents of 20-200 tokens; "
               "N=2^16, chain 60 + 29x40 bits + 4 special (60 bits), digits of 4 primes, inputs at level 3")


def fp64_scores(v, H, O):
    """Algorithm 1, steps 2-3 in FP64 (the reported accuracy check): s = (v H) O."""
    return (np.asarray(v, np.float64) @ H) @ O


def fasttext_measure(pft, torch, steps, warmup, plain_docs=1):
    from paper_1908_06972_gb300 import synth

    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, 60, 40, 60, 2.0 ** 40, SEED)
    tune(pft, ctx)
    n = 1 << LOGN
    t = n // 2
    pft.pft_keygen(ctx, [1 << i for i in range(15)], False)
    H, O = synth.fasttext_weights(77, FT_M, FT_N, FT_C)
    docs = synth.documents(78, FT_M, FT_BATCH)
    model = pft.pft_ft_model_create(ctx, H, O, FT_LEVEL)
    vs = []
    for d in range(FT_BATCH):
        pt = pft.pft_encode(ctx, docs[d], 2.0 ** 40, FT_LEVEL)
        vs.append(pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, 9000 + d))
        pft.pft_pt_destroy(pt)
    scores = [pft.pft_ct_create(ctx) for _ in range(FT_BATCH)]

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    batched = lambda: pft.pft_fasttext_infer_batch(ctx, model, vs, 1, scores)  # noqa: E731
    single = lambda: [pft.pft_fasttext_infer(ctx, model, [vs[d]], scores[d]) for d in range(4)]  # noqa: E731
    for _ in range(warmup):
        batched()
    tb = timed(batched, steps)
    single()
    ts = timed(single, 1)
    # accuracy of one document against the FP64 Algorithm 1
    dec = pft.pft_decrypt(ctx, scores[0])
    got = pft.pft_decode(ctx, dec, FT_C)[:FT_C].real
    pft.pft_pt_destroy(dec)
    err = float(np.max(np.abs(got - fp64_scores(docs[0], H, O))))
    # plain path: one library call per op per ciphertext
    Hp = [pft.pft_encode(ctx, H[:, j], 2.0 ** 40, FT_LEVEL) for j in range(FT_N)]
    Op = []
    for j in range(FT_N):
        row = np.zeros(FT_C)
        row[:] = O[j]
        Op.append(pft.pft_encode(ctx, row, 2.0 ** 40, FT_LEVEL - 1))
    tmp, rot, acc = pft.pft_ct_create(ctx), pft.pft_ct_create(ctx), pft.pft_ct_create(ctx)
    cols = [pft.pft_ct_create(ctx) for _ in range(FT_N)]

    def plain(d):
        for j in range(FT_N):
            pft.pft_mul_plain(ctx, vs[d], Hp[j], cols[j])
            for s in range(15):
                pft.pft_rotate(ctx, cols[j], 1 << s, rot)
                pft.pft_add(ctx, cols[j], rot, cols[j])
            pft.pft_rescale(ctx, cols[j], cols[j])
        pft.pft_mul_plain(ctx, cols[0], Op[0], acc)
        for j in range(1, FT_N):
            pft.pft_mul_plain(ctx, cols[j], Op[j], tmp)
            pft.pft_add(ctx, acc, tmp, acc)
        pft.pft_rescale(ctx, acc, acc)

    plain(0)
    tp = timed(lambda: [plain(d) for d in range(plain_docs)], 1)
    # rotation-light variant (diagonal packing, hoisted rotations; scores in slots 64 c)
    pft.pft_add_rotation_keys(ctx, list(range(1, FT_N)) + [FT_N << s for s in range(9)])
    dmodel = pft.pft_ft_model_create_diag(ctx, H, O, FT_LEVEL)
    dvs = []  # inputs at scale 2^50: this variant rotates the input before its plaintext product
    for d in range(FT_BATCH):
        pt = pft.pft_encode(ctx, docs[d], 2.0 ** 50, FT_LEVEL)
        dvs.append(pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, 9500 + d))
        pft.pft_pt_destroy(pt)
    dbatched = lambda: pft.pft_fasttext_infer_batch(ctx, dmodel, dvs, 1, scores)  # noqa: E731
    dbatched()
    tdb = timed(dbatched, steps)
    dec = pft.pft_decrypt(ctx, scores[0])
    dgot = pft.pft_decode(ctx, dec, t).real[[FT_N * cc for cc in range(FT_C)]]
    pft.pft_pt_destroy(dec)
    derr = float(np.max(np.abs(dgot - fp64_scores(docs[0], H, O))))
    pft.pft_ft_model_destroy(dmodel)
    for h in dvs:
        pft.pft_ct_destroy(h)
    for h in vs + scores + cols + [tmp, rot, acc]:
        pft.pft_ct_destroy(h)
    for h in Hp + Op:
        pft.pft_pt_destroy(h)
    pft.pft_ft_model_destroy(model)
    pft.pft_ctx_destroy(ctx)
    return {"workload": FT_WORKLOAD, "unit": "inferences/s",
            "batched_value": round(FT_BATCH * steps / tb, 3), "batch": FT_BATCH,
            "batch1_value": round(4 / ts, 3), "plain_value": round(plain_docs / tp, 3),
            "max_abs_err_vs_fp64": err, "rotations_per_inference": FT_N * 15,
            "diagonal_variant": {"batched_value": round(FT_BATCH * steps / tdb, 3), "max_abs_err_vs_fp64": derr,
                                 "rotations_per_inference": FT_N - 1 + 9 + 6, "input_scale": "2^50"}}


# Algorithmic mulmods of one key switch at level l (k special primes, digits of alpha primes, N =
# 2^16): transforms (l inverse, beta (l + k) - l forward for ModUp, 2k inverse and 2l forward for
# ModDown, N/2 log2 N butterflies each), ModUp conversion, inner product, ModDown conversion and
# scaling; the same count as the hot-path scope's per-unit figures.
def ks_mulmods(l, k=K_SP, alpha=ALPHA, logn=LOGN):
    n = 1 << logn
    E, beta = l + k, -(-l // alpha)
    digits = [min(alpha, l - j * alpha) for j in range(beta)]
    n_ntt = l + sum(E - a for a in digits) + 2 * k + 2 * l
    return n * (n_ntt * logn / 2 + sum(digits) + sum(a * (E - a) for a in digits) + 2 * beta * E + 2 * (k + k * l + l))


def fasttext_mulmods(l, cols=FT_N, logn=LOGN):
    """One Fig. 3 inference at level l: cols column products, log2(N/2) rotations per column
    (TotalSum), a rescale per column, the output products and a final rescale."""
    n = 1 << logn
    rot = ks_mulmods(l)  # a rotation's automorphism and the TotalSum additions take no mulmods
    rescale = lambda lv: 2 * (lv * (n // 2) * logn + (lv - 1) * n)  # noqa: E731
    return cols * (2 * l * n + (logn - 1) * rot + rescale(l)) + cols * 2 * (l - 1) * n + rescale(l - 1)


def fasttext_measure_l30(pft, torch, level=30, batch=8):
    """The fastText inference at the top of the 30-prime chain: batch `batch` and batch 1 of the
    Fig. 3 sequence (960 rotations per inference) and 32 documents of the rotation-light one."""
    from paper_1908_06972_gb300 import synth

    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, 60, 40, 60, 2.0 ** 40, SEED)
    tune(pft, ctx)
    pft.pft_keygen(ctx, [1 << i for i in range(15)], False)
    H, O = synth.fasttext_weights(77, FT_M, FT_N, FT_C)
    docs = synth.documents(78, FT_M, FT_BATCH)
    t = (1 << LOGN) // 2

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def enc(d, scale, nonce):
        pt = pft.pft_encode(ctx, docs[d], scale, level)
        h = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, nonce)
        pft.pft_pt_destroy(pt)
        return h

    model = pft.pft_ft_model_create(ctx, H, O, level)
    vs = [enc(d, 2.0 ** 40, 9100 + d) for d in range(batch)]
    scores = [pft.pft_ct_create(ctx) for _ in range(FT_BATCH)]
    batched = lambda: pft.pft_fasttext_infer_batch(ctx, model, vs, 1, scores[:batch])  # noqa: E731
    batched()
    tb = timed(batched)
    ts = timed(lambda: pft.pft_fasttext_infer(ctx, model, [vs[0]], scores[0]))
    dec = pft.pft_decrypt(ctx, scores[0])
    err = float(np.max(np.abs(pft.pft_decode(ctx, dec, FT_C)[:FT_C].real - fp64_scores(docs[0], H, O))))
    pft.pft_pt_destroy(dec)
    for h in vs:
        pft.pft_ct_destroy(h)
    pft.pft_ft_model_destroy(model)
    pft.pft_add_rotation_keys(ctx, list(range(1, FT_N)) + [FT_N << s for s in range(9)])
    dmodel = pft.pft_ft_model_create_diag(ctx, H, O, level)
    dvs = [enc(d, 2.0 ** 50, 9600 + d) for d in range(FT_BATCH)]
    dbatched = lambda: pft.pft_fasttext_infer_batch(ctx, dmodel, dvs, 1, scores)  # noqa: E731
    dbatched()
    tdb = timed(dbatched)
    dec = pft.pft_decrypt(ctx, scores[0])
    derr = float(np.max(np.abs(pft.pft_decode(ctx, dec, t).real[[FT_N * cc for cc in range(FT_C)]]
                               - fp64_scores(docs[0], H, O))))
    pft.pft_pt_destroy(dec)
    for h in dvs + scores:
        pft.pft_ct_destroy(h)
    pft.pft_ft_model_destroy(dmodel)
    pft.pft_ctx_destroy(ctx)
    mm = fasttext_mulmods(level)
    return {"level": level, "unit": "inferences/s", "batched_value": round(batch / tb, 3), "batch": batch,
            "batch1_value": round(1 / ts, 3), "max_abs_err_vs_fp64": err,
            "gmulmod_per_inference": round(mm / 1e9, 1), "batched_gmulmod_s": round(mm * batch / tb / 1e9, 1),
            "diagonal_variant": {"batched_value": round(FT_BATCH / tdb, 3), "batch": FT_BATCH,
                                 "max_abs_err_vs_fp64": derr, "input_scale": "2^50"}}


# ---- serving loop: Poisson arrivals, continuous batching ------------------------------------------
SV_RINGS = [  # (log_n, limbs, special primes, primes per digit, request levels)
    (16, 30, 4, 4, (12, 30)),
    (15, 18, 2, 2, (12, 18)),
]
SV_WORKLOAD = ("Poisson arrivals of encrypted fastText inferences (vocab 32768, dim 64, 14 classes); two rings, half "
               "the requests each: N=2^16 (60 + 29x40 bits + 4 special, digits of 4; request levels U{12..30}; "
               "vocabulary in 1 ciphertext) and N=2^15 (60 + 17x40 bits + 2 special, digits of 2; U{12..18}, "
               "vocabulary in 2 ciphertexts); keys and models resident; inputs and scores in host memory")


def serve_measure(pft, torch, n_req, rate, budget_gib, near, fig3_leg=True, seed=31):
    """Serving legs: the rotation-light sequence on both rings (diagonal packing; per vocabulary
    chunk on the N=2^15 ring; inputs at 2^50) saturated at `rate`, then offered at `near` times
    the measured capacity; and (fig3_leg) the Fig. 3 sequence (960 rotations per inference at
    N=2^16, inputs at 2^40) saturated, for comparison."""
    from paper_1908_06972_gb300 import serving, synth

    H, O = synth.fasttext_weights(77, FT_M, FT_N, FT_C)
    streams, ctxs = [], []
    for logn, lim, ksp, alpha, _ in SV_RINGS:
        st = torch.cuda.Stream()
        ctx = pft.pft_ctx_create(logn, lim, ksp, alpha, 60, 40, 60, 2.0 ** 40, SEED, stream=st.cuda_stream)
        tune(pft, ctx)
        steps = [1 << i for i in range(logn - 1)] + list(range(3, FT_N))  # TotalSum; diagonal shifts 1..n-1
        pft.pft_keygen(ctx, steps, False)
        streams.append(st)
        ctxs.append(ctx)
    torch.cuda.synchronize()
    seqs = {"rotation_light": ([pft.pft_ft_model_create_diag(c, H, O, r[1]) for c, r in zip(ctxs, SV_RINGS)],
                               2.0 ** 50, [[FT_N * cc for cc in range(FT_C)]] * len(SV_RINGS))}
    if fig3_leg:
        seqs["fig3"] = ([pft.pft_ft_model_create(c, H, O, r[1]) for c, r in zip(ctxs, SV_RINGS)], 2.0 ** 40,
                        [list(range(FT_C))] * len(SV_RINGS))

    def trace(count, rate_, tseed, scale):
        rng = np.random.default_rng(tseed)
        times = serving.poisson_arrivals(rate_, count, tseed)
        docs = synth.documents(tseed + 1, FT_M, count)
        reqs = []
        for i in range(count):
            r = int(rng.integers(0, 2))
            logn, _, _, _, (lo, hi) = SV_RINGS[r]
            level = int(rng.integers(lo, hi + 1))
            n, t = 1 << logn, 1 << (logn - 1)
            chunks = -(-FT_M // t)
            coeffs = np.zeros((chunks, 2, level, n), np.uint64)
            for c in range(chunks):
                pt = pft.pft_encode(ctxs[r], docs[i][c * t:(c + 1) * t], scale, level)
                ct = pft.pft_encrypt(ctxs[r], pt, pft.PFT_ENC_SK, 40000 + 4 * i + c)
                pft.pft_ct_export(ctxs[r], ct, coeffs[c])
                pft.pft_ct_destroy(ct)
                pft.pft_pt_destroy(pt)
            out = np.zeros((2, level - 2, n), np.uint64)
            reqs.append(serving.Request(t=float(times[i]), ring=r, level=level, scale=scale, coeffs=coeffs,
                                        out=out, tag=i))
        return reqs, docs

    def run(models, reqs):
        srv = pft.pft_server_create(ctxs, models, int(budget_gib * 2 ** 30))
        try:
            return serving.replay(srv, reqs)
        finally:
            pft.pft_server_destroy(srv)

    def summary(res, reqs, rate_):
        return {"requests": len(reqs), "offered_rate": round(rate_, 3), "throughput": round(res.throughput(), 3),
                "p50_s": round(res.percentile(50), 3), "p99_s": round(res.percentile(99), 3),
                "makespan_s": round(res.makespan, 3), "max_active": res.max_active, "iterations": res.iterations,
                "peak_resident_gib": round(res.peak_bytes / 2 ** 30, 2),
                "requests_per_ring": [sum(1 for q in reqs if q.ring == r) for r in range(len(SV_RINGS))],
                "mean_level": round(float(np.mean([q.level for q in reqs])), 2)}

    def accuracy(res, reqs, docs, slots):
        """Decrypt the first request of each ring against FP64 Algorithm 1."""
        err = 0.0
        for r in range(len(SV_RINGS)):
            q = next((q for q in reqs if q.ring == r), None)
            if q is None:
                continue
            h = pft.pft_ct_import(ctxs[r], q.out, res.done[q.tag]["scale"])
            dec = pft.pft_decrypt(ctxs[r], h)
            got = pft.pft_decode(ctxs[r], dec, 1 << (SV_RINGS[r][0] - 1)).real[slots[r]]
            pft.pft_pt_destroy(dec)
            pft.pft_ct_destroy(h)
            err = max(err, float(np.max(np.abs(got - fp64_scores(docs[q.tag], H, O)))))
        return err

    out = {"workload": SV_WORKLOAD, "unit": "inferences/s", "budget_gib": budget_gib}
    for name, (models, scale, slots) in seqs.items():
        warm, _ = trace(2, 1000.0, seed + 100, scale)  # kernels loaded, allocator pools grown
        run(models, warm)
        reqs, docs = trace(n_req, rate, seed, scale)
        res = run(models, reqs)
        leg = {"saturated": summary(res, reqs, rate), "max_abs_err_vs_fp64": accuracy(res, reqs, docs, slots)}
        if name == "rotation_light" and near > 0:
            rate_near = near * res.throughput()
            reqs_n, _ = trace(n_req, rate_near, seed + 7, scale)
            leg["near_capacity"] = summary(run(models, reqs_n), reqs_n, rate_near)
        out[name] = leg
        for m in models:
            pft.pft_ft_model_destroy(m)
    for c in ctxs:
        pft.pft_ctx_destroy(c)
    return out


# ---- primitive operations at the top level ----------------------------------------------------
OPS_WORKLOAD = ("the benchmark chain (N=2^16, 60 + 29x50 bits + 4 special primes of 60 bits, about 1750 bits of "
                "modulus, 128-bit) at its top level 30: one ciphertext per call, and 64 per batched call")


def ops_measure(pft, torch, synth, ctx, reps):
    """Latency of each primitive for one ciphertext at level 30 and the time per ciphertext of
    the batched call over 64, with CUDA events around `reps` calls after a warm-up."""
    L_TOP, NB = L, 64
    pts, cts = [], []

    def enc(seed, nonce):
        pt = pft.pft_encode(ctx, synth.slots(seed, 256), SCALE, L_TOP)
        h = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, nonce)
        pft.pft_pt_destroy(pt)
        cts.append(h)
        return h

    A = [enc(7000 + i, 9000 + 2 * i) for i in range(NB)]
    B = [enc(8000 + i, 9001 + 2 * i) for i in range(NB)]
    P = [pft.pft_encode(ctx, synth.slots(9500 + i, 256), SCALE, L_TOP) for i in range(NB)]
    pts += P
    C = [pft.pft_ct_create(ctx) for _ in range(NB)]
    D = [pft.pft_ct_create(ctx) for _ in range(NB)]
    cts += C + D
    pft.pft_mul_relin_batch(ctx, A, B, C)  # C at level 30 with the product's scale, for rescale

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    one = {"hmul_relin": lambda: pft.pft_mul_relin(ctx, A[0], B[0], D[0]),
           "hmulplain": lambda: pft.pft_mul_plain(ctx, A[0], P[0], D[0]),
           "haddplain": lambda: pft.pft_add_plain(ctx, A[0], P[0], D[0]),
           "rescale": lambda: pft.pft_rescale(ctx, C[0], D[0]),
           "rotate": lambda: pft.pft_rotate(ctx, A[0], 1, D[0])}
    many = {"hmul_relin": lambda: pft.pft_mul_relin_batch(ctx, A, B, D),
            "hmulplain": lambda: pft.pft_mul_plain_batch(ctx, A, P, D),
            "rescale": lambda: pft.pft_rescale_batch(ctx, C, D),
            "rotate": lambda: pft.pft_rotate_batch(ctx, A, 1, D)}
    lat = {k: round(timed(f), 4) for k, f in one.items()}
    per = {k: round(timed(f) / NB, 4) for k, f in many.items()}
    for h in cts:
        pft.pft_ct_destroy(h)
    for p in pts:
        pft.pft_pt_destroy(p)
    return {"workload": OPS_WORKLOAD, "unit": "ms", "level": L_TOP, "latency_one_ciphertext_ms": lat,
            "per_ciphertext_in_batch_of_64_ms": per,
            "hmul_relin_per_s": {"one_at_a_time": round(1e3 / lat["hmul_relin"], 1),
                                 "batched": round(1e3 / per["hmul_relin"], 1)}}


# ---- persistent job queue over two rings ------------------------------------------------------
QU_WORKLOAD = ("64 ciphertexts at N=2^16 (60 + 29x50-bit chain, levels U{5..30}) and 64 at N=2^15 "
               "(60 + 17x40-bit chain, levels U{12..18}): per ciphertext one HADD and one HMULPLAIN "
               "(plaintext at the ciphertext's level), all in one list")


def queue_measure(pft, torch, reps):
    """One pft_run_jobs launch over both rings against the per-ring batched calls (one launch
    per op and ring); GB/s of algorithmic bytes (HADD 48, HMULPLAIN 40 bytes per coefficient
    and limb) against the measured HBM copy rate."""
    from paper_1908_06972_gb300 import synth

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    rng = np.random.default_rng(77)
    rings = [(16, 30, 4, 4, 60, 50, 60, rng.integers(5, 31, 64)), (15, 18, 2, 2, 60, 40, 60, rng.integers(12, 19, 64))]
    ctxs, rows, handles, pts = [], [], [], []
    for logn, L, k, alpha, f, m, sp, lv in rings:
        ctx = pft.pft_ctx_create(logn, L, k, alpha, f, m, sp, 2.0 ** 40, (0x9E, logn, 1, 2))
        pft.pft_keygen(ctx, [], False)  # the secret key only: nothing here switches keys
        ctxs.append(ctx)
        r = []
        def enc(z, nonce, level):
            pt = pft.pft_encode(ctx, z, 2.0 ** 40, level)
            h = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, nonce)
            pft.pft_pt_destroy(pt)
            return h

        for i, l in enumerate(lv):
            l = int(l)
            x, y = enc(synth.slots(i, 64), 2 * i, l), enc(synth.slots(i + 500, 64), 2 * i + 1, l)
            p = pft.pft_encode(ctx, synth.slots(i + 900, 64), 2.0 ** 20, l)
            o1, o2 = pft.pft_ct_create(ctx), pft.pft_ct_create(ctx)
            handles += [x, y, o1, o2]
            pts.append(p)
            r.append((x, y, p, o1, o2, l, 1 << logn))
        rows.append(r)
    jobs = []
    nbytes = 0.0
    for r in rows:
        for x, y, p, o1, o2, l, n in r:
            jobs.append(dict(op=pft.PFT_JOB_ADD, a=x, b=y, out=o1))
            jobs.append(dict(op=pft.PFT_JOB_MUL_PLAIN, a=x, p=p, out=o2))
            nbytes += (48 + 40) * l * n

    def per_ring():
        for ctx, r in zip(ctxs, rows):
            pft.pft_add_batch(ctx, [e[0] for e in r], [e[1] for e in r], [e[3] for e in r])
            pft.pft_mul_plain_batch(ctx, [e[0] for e in r], [e[2] for e in r], [e[4] for e in r])

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_q = timed(lambda: pft.pft_run_jobs(ctxs[0], jobs))
    pft.pft_device_status(ctxs[0])
    t_r = timed(per_ring)
    for h in handles:
        pft.pft_ct_destroy(h)
    for p in pts:
        pft.pft_pt_destroy(p)
    for c in ctxs:
        pft.pft_ctx_destroy(c)
    gbs_q, gbs_r = nbytes / t_q / 1e9, nbytes / t_r / 1e9
    return {"workload": QU_WORKLOAD, "jobs": len(jobs), "algorithmic_gb": round(nbytes / 1e9, 3),
            "one_launch_ms": round(1e3 * t_q, 3), "per_ring_batched_ms": round(1e3 * t_r, 3),
            "roofline": {"bound": "hbm", "kernel": "k_job_queue", "achieved": round(gbs_q, 1),
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(gbs_q / peaks["hbm_gbs"], 4)},
            "per_ring_gbs": round(gbs_r, 1)}


# ---- encrypted minibatch training (Sec. 4.2, Algorithm 5) -----------------------------------------
TR_M, TR_N, TR_C, TR_L, TR_ETA = 8192, 32, 4, 30, 0.25
TR_WORKLOAD = ("encrypted fastText training step: vocab 8192 (one N=2^16 ciphertext), dim 32, 4 classes, "
               "Zipf(1.1) documents, one-hot labels; forward with the paper's softmax polynomial, homomorphic "
               "backward, one SGD update; chain 60 + 29x40 bits + 4 special (60 bits), digits of 4, model at level 30")


def fp64_train_grads(V, Y, H, O):
    """Gradients of L = sum [s^3/24 + s^2/4 + s/4 - y s], s = V H O, in FP64 (the reported
    accuracy check): g = s^2/8 + s/2 + 1/4 - y, dH = V^T (g O^T), dO = (V H)^T g."""
    Hh = V @ H
    S = Hh @ O
    G = S * S / 8 + S / 2 + 0.25 - Y
    return V.T @ (G @ O.T), Hh.T @ G


TR_LIFT = 10


def train_diag(pft, ctx, enc, new, dec, timed, H, O, V, Y, ref_H, ref_O, sc, n_docs):
    """The same minibatch in the rotation-light layout: the n diagonals D_k[i] = H[(i+k) mod t,
    i mod n], P[n c + j] = O[j, c] one level below, a mask of the score slots n c at 2^-10 times
    the scale (the documents are lifted by 2^10 before their rotations), labels over the class
    blocks; the gradients come back as the diagonals of dH and dO in the layout of P."""
    t = (1 << LOGN) // 2
    n = TR_N
    pft.pft_add_rotation_keys(ctx, [k for k in range(1, n) if k & (k - 1)] + [-(1 << s) for s in range(n.bit_length() - 1)])
    Hp = np.zeros((t, n))
    Hp[:TR_M] = H
    i = np.arange(t)
    Dv = [Hp[(i + k) % t, i % n] for k in range(n)]
    Pv = np.zeros(t)
    Mv = np.zeros(t)
    for cc in range(TR_C):
        Pv[n * cc:n * cc + n] = O[:, cc]
        Mv[n * cc] = 1.0
    Dc = [enc(Dv[k], TR_L, sc, 3000 + k) for k in range(n)]
    Pc = enc(Pv, TR_L - 1, sc, 3100)
    mask = pft.pft_encode(ctx, Mv, sc / 2.0 ** TR_LIFT, TR_L)
    model = pft.pft_ft_enc_model_create_diag(ctx, Dc, Pc, mask, TR_M, n, TR_C, TR_LIFT)
    dl, ll, ls = pft.pft_fasttext_train_spec(ctx, model, sc)
    pad = np.zeros((n_docs, t))
    pad[:, :TR_M] = V
    docs = [enc(pad[b], dl, sc, 4000 + b) for b in range(n_docs)]
    labels = []
    for b in range(n_docs):
        w = np.zeros(t)
        w[:n * TR_C] = np.repeat(Y[b] - 0.25, n)
        labels.append(enc(w, ll, ls, 5000 + b))
    gD = [new() for _ in range(n)]
    gP = [new()]
    warm = pft.pft_ft_enc_model_create_diag(ctx, Dc, Pc, mask, TR_M, n, TR_C, TR_LIFT)
    pft.pft_fasttext_train_step(ctx, warm, docs[:2], labels[:2], TR_ETA, gD, gP)
    pft.pft_ft_enc_model_destroy(warm)
    t_step = timed(lambda: pft.pft_fasttext_train_step(ctx, model, docs, labels, TR_ETA, gD, gP))
    Gp = np.zeros((t, n))
    Gp[:TR_M] = ref_H
    err = 0.0
    for k in range(n):
        err = max(err, float(np.max(np.abs(dec(gD[k], t) - Gp[(i + k) % t, i % n]))))
    got_P = dec(gP[0], n * TR_C)
    err = max(err, float(np.max(np.abs(got_P.reshape(TR_C, n).T - ref_O))))
    lv = pft.pft_ft_enc_model_levels(model)
    pft.pft_ft_enc_model_destroy(model)
    pft.pft_pt_destroy(mask)
    rots = (n - 1) + 2 * (LOGN - 1 - (n.bit_length() - 1)) + 2 * (n.bit_length() - 1)
    return {"step_s": round(t_step, 3), "ms_per_doc": round(1e3 * t_step / n_docs, 2), "rotations_per_doc": rots,
            "max_abs_err_grad_vs_fp64": err, "model_levels_after": list(lv),
            "lift_bits": TR_LIFT,
            "layout": "diagonals of H (n ciphertexts), O packed in one ciphertext, score mask; not in the paper"}


def train_measure(pft, torch, n_docs, plain_docs, with_diag=True):
    from paper_1908_06972_gb300 import synth

    sc = 2.0 ** 40
    ctx = pft.pft_ctx_create(LOGN, TR_L, K_SP, ALPHA, 60, 40, 60, sc, SEED)
    tune(pft, ctx)
    pft.pft_keygen(ctx, [1 << i for i in range(LOGN - 1)], True)
    t = (1 << LOGN) // 2
    handles = []

    def enc(z, level, scale, nonce):
        pt = pft.pft_encode(ctx, z, scale, level)
        h = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, nonce)
        pft.pft_pt_destroy(pt)
        handles.append(h)
        return h

    def new():
        h = pft.pft_ct_create(ctx)
        handles.append(h)
        return h

    def dec(h, k):
        pt = pft.pft_decrypt(ctx, h)
        z = pft.pft_decode(ctx, pt, k).real
        pft.pft_pt_destroy(pt)
        return z

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    H, O = synth.fasttext_weights(61, TR_M, TR_N, TR_C)
    V = synth.documents(62, TR_M, n_docs)
    Y = np.eye(TR_C)[np.random.default_rng(63).integers(0, TR_C, n_docs)]
    Hc = [enc(H[:, j], TR_L, sc, 10 + j) for j in range(TR_N)]
    Oc = [enc(O[j], TR_L - 1, sc, 100 + j) for j in range(TR_N)]
    model = pft.pft_ft_enc_model_create(ctx, Hc, Oc, TR_M, TR_N, TR_C)
    dl, ll, ls = pft.pft_fasttext_train_spec(ctx, model, sc)
    docs = [enc(V[b], dl, sc, 1000 + b) for b in range(n_docs)]
    labels = [enc(Y[b] - 0.25, ll, ls, 2000 + b) for b in range(n_docs)]
    gH = [new() for _ in range(TR_N)]
    gO = [new() for _ in range(TR_N)]
    warm = pft.pft_ft_enc_model_create(ctx, Hc, Oc, TR_M, TR_N, TR_C)
    pft.pft_fasttext_train_step(ctx, warm, docs[:2], labels[:2], TR_ETA, gH, gO)
    pft.pft_ft_enc_model_destroy(warm)
    t_step = timed(lambda: pft.pft_fasttext_train_step(ctx, model, docs, labels, TR_ETA, gH, gO))
    ref_H, ref_O = fp64_train_grads(V, Y, H, O)
    got_H = np.stack([dec(gH[j], TR_M) for j in range(TR_N)], 1)
    got_O = np.stack([dec(gO[j], TR_C) for j in range(TR_N)])
    err = float(max(np.max(np.abs(got_H - ref_H)), np.max(np.abs(got_O - ref_O))))
    lvH, lvO = pft.pft_ft_enc_model_levels(model)
    pft.pft_ft_enc_model_destroy(model)

    # plain path: one library call per operation per ciphertext (products relinearised one by
    # one), on `plain_docs` documents, then the same update
    def plain(nd):
        n = TR_N
        accO, accH = [None] * n, [None] * n
        tmp = new()
        for b in range(nd):
            v, w = docs[b], labels[b]
            hs = []
            for j in range(n):
                T = new()
                pft.pft_mul_relin(ctx, v, Hc[j], T)
                st = 1
                while st < t:
                    pft.pft_rotate(ctx, T, st, tmp)
                    pft.pft_add(ctx, T, tmp, T)
                    st *= 2
                pft.pft_rescale(ctx, T, T)
                hs.append(T)
            S = new()
            for j in range(n):
                pft.pft_mul_relin(ctx, hs[j], Oc[j], tmp if j else S)
                if j:
                    pft.pft_add(ctx, S, tmp, S)
            pft.pft_rescale(ctx, S, S)
            U = new()
            pft.pft_add_const(ctx, S, 2.0, U)
            pft.pft_mul_relin(ctx, U, U, U)
            pft.pft_rescale(ctx, U, U)
            pft.pft_ct_set_scale(U, 8.0 * pft.pft_ct_scale(U))
            pft.pft_add_const(ctx, U, -0.5, U)
            g = new()
            pft.pft_sub(ctx, U, w, g)
            lg = pft.pft_ct_level(g)
            for j in range(n):
                a, bb, P = new(), new(), new()
                pft.pft_drop_level(ctx, hs[j], lg, a)
                pft.pft_mul_relin(ctx, a, g, P)
                if accO[j] is None:
                    accO[j] = P
                else:
                    pft.pft_add(ctx, accO[j], P, accO[j])
                pft.pft_drop_level(ctx, Oc[j], lg, bb)
                E = new()
                pft.pft_mul_relin(ctx, g, bb, E)
                st = 1
                while st < t:
                    pft.pft_rotate(ctx, E, st, tmp)
                    pft.pft_add(ctx, E, tmp, E)
                    st *= 2
                pft.pft_rescale(ctx, E, E)
                vd, P2 = new(), new()
                pft.pft_drop_level(ctx, v, pft.pft_ct_level(E), vd)
                pft.pft_mul_relin(ctx, vd, E, P2)
                if accH[j] is None:
                    accH[j] = P2
                else:
                    pft.pft_add(ctx, accH[j], P2, accH[j])
        for j in range(n):
            pft.pft_rescale(ctx, accO[j], accO[j])
            pft.pft_rescale(ctx, accH[j], accH[j])
        return accH, accO

    t_plain = None
    if plain_docs > 0:
        t_plain = timed(lambda: plain(plain_docs))
    diag = train_diag(pft, ctx, enc, new, dec, timed, H, O, V, Y, ref_H, ref_O, sc, n_docs) if with_diag else None
    for h in handles:
        pft.pft_ct_destroy(h)
    pft.pft_ctx_destroy(ctx)
    return {"workload": TR_WORKLOAD, "docs": n_docs, "unit": "s per training step", "rotation_light": diag,
            "step_s": round(t_step, 3), "ms_per_doc": round(1e3 * t_step / n_docs, 2),
            "rotations_per_doc": 2 * TR_N * (LOGN - 1),
            "plain": None if t_plain is None else {
                "docs_timed": plain_docs, "ms_per_doc": round(1e3 * t_plain / plain_docs, 2),
                "step_s_extrapolated": round(t_plain / plain_docs * n_docs, 3),
                "note": "one call per operation per ciphertext, products relinearised one by one, "
                        "update not included"},
            "max_abs_err_grad_vs_fp64": err, "model_levels_after": [lvH, lvO], "eta": TR_ETA}


AUTOTUNE = [True]  # --autotune 0: every context keeps the plans it starts with


def tune(pft, ctx):
    """The transform-plan search on a leg's context, as a user would run it (unless disabled)."""
    if AUTOTUNE[0]:
        pft.pft_autotune(ctx)


def link_rates(host_in, host_out, reps=5):
    """Host <-> device copy rates (GB/s, best of `reps`) of one page-locked input and one output
    buffer of the end-to-end leg, timed with CUDA events on a stream of their own: the bound the
    end-to-end figure meets when its copies take longer than a step's compute."""
    import torch

    st = torch.cuda.Stream()
    dev = torch.empty(max(host_in.nbytes, host_out.nbytes) // 8, dtype=torch.int64, device="cuda")
    src = torch.from_numpy(host_in.view(np.int64)).view(-1)
    dst = torch.from_numpy(host_out.view(np.int64)).view(-1)
    best = {"h2d": 0.0, "d2h": 0.0}
    with torch.cuda.stream(st):
        for _ in range(reps):
            for key, fn, nbytes in (("h2d", lambda: dev[:src.numel()].copy_(src, non_blocking=True), host_in.nbytes),
                                    ("d2h", lambda: dst.copy_(dev[:dst.numel()], non_blocking=True), host_out.nbytes)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                e1.synchronize()
                best[key] = max(best[key], nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dev
    return {key: round(v, 1) for key, v in best.items()}


# ---- isolated kernel case (for ncu captures and burst rooflines) --------------------------------

def run_case_ntt(args):
    """Forward + inverse transform of 16 polynomials x 30 limbs at N = 2^16 (252 MB > L2)."""
    import torch

    import paper_1908_06972_gb300 as pft

    torch.cuda.set_device(0)
    pft.build()
    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, FIRST, MID, SPECIAL, SCALE, SEED)
    n, polys = 1 << LOGN, 16
    primes = pft.pft_ctx_info(ctx)["primes"]
    rng = np.random.default_rng(3)
    host = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes[:L]]) for _ in range(polys)])
    t = torch.from_numpy(host.view(np.int64)).cuda()
    for _ in range(args.warmup):
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 0)
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 1)
    torch.cuda.synchronize()
    pft.pft_prof_start("ntt.fwd")
    for _ in range(args.steps):
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 0)
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 1)
    fwd_ms, fwd_n, _, fwd_work = pft.pft_prof_stop()
    pft.pft_prof_start("ntt.inv")
    for _ in range(args.steps):
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 0)
        pft.pft_ntt(ctx, t.data_ptr(), polys, L, 1)
    inv_ms, inv_n, _, inv_work = pft.pft_prof_stop()
    torch.cuda.synchronize()
    ok = bool(np.array_equal(t.cpu().numpy().view(np.uint64), host))
    lo, hi, wide = pft.pft_mul_rates(ctx)
    peak = alu_bound(lo, min(hi, wide))
    bytes_per_pass = polys * L * n * 8 * 2
    res = {"case": "ntt", "polys": polys, "limbs": L, "N": n, "round_trip_exact": ok,
           "fwd_us_per_pass": round(1e3 * fwd_ms / fwd_n, 2), "inv_us_per_pass": round(1e3 * inv_ms / inv_n, 2),
           "fwd_gmulmod_s": round(fwd_work / (fwd_ms / 1e3) / 1e9, 1),
           "inv_gmulmod_s": round(inv_work / (inv_ms / 1e3) / 1e9, 1),
           "alu_peak_gmulmod_s": round(peak / 1e9, 1),
           "fwd_gbs": round(bytes_per_pass * fwd_n / (fwd_ms / 1e3) / 1e9, 1),
           "inv_gbs": round(bytes_per_pass * inv_n / (inv_ms / 1e3) / 1e9, 1)}
    print(json.dumps(res))
    pft.pft_ctx_destroy(ctx)


def run_case_ks(args):
    """Batched HMUL + relinearisation of 4 ciphertext pairs at level 30 (the benchmark's chain)."""
    import torch

    import paper_1908_06972_gb300 as pft
    from paper_1908_06972_gb300 import synth

    torch.cuda.set_device(0)
    pft.build()
    ctx = pft.pft_ctx_create(LOGN, L, K_SP, ALPHA, FIRST, MID, SPECIAL, SCALE, SEED,
                             flags=pft.PFT_COMPRESSED_KEYS if args.compressed_keys else 0)
    pft.pft_keygen(ctx, [], True)
    A, B = [], []
    for i in range(4):
        p = pft.pft_encode(ctx, synth.slots(i, 64), SCALE, L)
        A.append(pft.pft_encrypt(ctx, p, pft.PFT_ENC_SK, 2 * i))
        B.append(pft.pft_encrypt(ctx, p, pft.PFT_ENC_SK, 2 * i + 1))
        pft.pft_pt_destroy(p)
    C = [pft.pft_ct_create(ctx) for _ in range(4)]
    for _ in range(args.warmup):
        pft.pft_mul_relin_batch(ctx, A, B, C)
    torch.cuda.synchronize()
    res = {"case": "ks", "level": L, "batch": 4, "compressed_keys": bool(args.compressed_keys)}
    for fam in ("bconv", "ks_inner", "ntt", "epi", "sub_scale"):
        pft.pft_prof_start(fam)
        for _ in range(args.steps):
            pft.pft_mul_relin_batch(ctx, A, B, C)
        ms, n, tot, work = pft.pft_prof_stop()
        res[fam] = {"us_per_launch": round(1e3 * ms / max(1, n), 2), "launches_per_op": n // args.steps,
                    "gbs": round(work / (ms / 1e3) / 1e9, 1) if work and fam not in ("ntt", "epi") else None}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pft.pft_mul_relin_batch(ctx, A, B, C)
    e1.record()
    torch.cuda.synchronize()
    res["ms_per_batch"] = round(e0.elapsed_time(e1) / args.steps, 3)
    print(json.dumps(res))
    for h in A + B + C:
        pft.pft_ct_destroy(h)
    pft.pft_ctx_destroy(ctx)


# ---- CPU oracle -------------------------------------------------------------------------------------
_ORACLES = {}


def _oracle_at(level):
    """Oracle on the chain truncated at `level` (the slice of the full keys a level-`level`
    ciphertext touches), with its keys and two input ciphertexts; built once per level."""
    if level not in _ORACLES:
        from oracle import ckks
        from paper_1908_06972_gb300 import synth

        orc = ckks.Oracle(LOGN, level, K_SP, ALPHA, FIRST, MID, SPECIAL, SCALE, SEED)
        orc.keygen([1], True)
        a = orc.encrypt_sk(orc.encode(synth.slots(1, 256), level=level), 1)
        b = orc.encrypt_sk(orc.encode(synth.slots(2, 256), level=level), 2)
        _ORACLES[level] = (orc, a, b)
    return _ORACLES[level]


def cpu_baseline(levels_spec):
    """The oracle on a bounded sample of the workload: one ciphertext pair at each sampled
    level through mul_relin and one rotation; the time of a unit (mul_relin + 16 rotations) is
    interpolated linearly in the level between the samples and averaged over the workload's
    64 levels."""
    pts = sorted(int(x) for x in str(levels_spec).split(","))
    unit, measured = [], 0.0
    for lv in pts:
        orc, a, b = _oracle_at(lv)
        t0 = time.perf_counter()
        c = orc.mul_relin(a, b)
        t1 = time.perf_counter()
        orc.rotate(c, 1)
        t2 = time.perf_counter()
        unit.append((t1 - t0) + 16 * (t2 - t1))
        measured += t2 - t0
    wl = levels()
    unit_s = float(np.mean(np.interp(wl, pts, unit)))
    cores = len(os.sched_getaffinity(0))
    return {"value": round(1.0 / unit_s, 6), "unit": "mult+relin/s", "cores": cores, "kind": "oracle",
            "sample": "one ciphertext pair at each of levels %s through mul_relin + 1 rotation (%.1f s measured); "
                      "unit time (mul_relin + 16 rotations) interpolated in the level and averaged over the "
                      "workload's 64 levels (mean %.2f)" % (", ".join(map(str, pts)), measured, float(np.mean(wl)))}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    times = []
    for _ in range(args.warmup):
        cpu_baseline(args.cpu_level)
    for _ in range(args.steps):
        r = cpu_baseline(args.cpu_level)
        times.append(1.0 / r["value"])
    value = len(times) / sum(times)
    # a step is the whole batch of 64 units; the oracle is timed on a sample and extrapolated
    out = {"impl": "reference", "metric": "HE mult+relin/s at N=2^16; enc. fastText inferences/s, batched vs plain",
           "value": round(value, 6), "unit": "mult+relin/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * BATCH * sum(times) / len(times), 1),
           "ms_per_unit": round(1e3 * sum(times) / len(times), 1), "extrapolated": True,
           "sampled_levels": [int(x) for x in str(args.cpu_level).split(",")],
           "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "batch": BATCH},
           "cpu_baseline": {"value": round(value, 6), "unit": "mult+relin/s", "kind": "oracle",
                            "cores": len(os.sched_getaffinity(0)), "sample": r["sample"]},
           "e2e": {"value": round(value, 6), "unit": "mult+relin/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--autotune", type=int, default=1,
                    help="0: no transform-plan search; the contexts' initial plans (for ncu captures)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--roofline-kernel", default="ntt")
    ap.add_argument("--cpu-level", default="5,19,30", help="levels the CPU oracle is timed at")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="step", choices=["step", "ntt", "ks"])
    ap.add_argument("--fasttext", type=int, default=1, help="also measure encrypted fastText inference")
    ap.add_argument("--graph", type=int, default=1, help="also measure the step as one CUDA-graph launch")
    ap.add_argument("--fasttext-l30", type=int, default=1, help="also measure fastText at level 30")
    ap.add_argument("--compressed-keys", action="store_true",
                    help="seeded compressed switching keys (the step and --case ks)")
    ap.add_argument("--train", type=int, default=64, help="documents per encrypted training step (0: skip)")
    ap.add_argument("--train-plain-docs", type=int, default=2, help="documents timed on the plain training path")
    ap.add_argument("--train-diag", type=int, default=1, help="also time the rotation-light training layout (0: skip)")
    ap.add_argument("--queue", type=int, default=10, help="repetitions of the two-ring job-queue leg (0: skip)")
    ap.add_argument("--ops", type=int, default=20, help="repetitions of each primitive at the top level (0: skip)")
    ap.add_argument("--serve", type=int, default=96, help="requests in the serving trace (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="offered load of the serving trace (req/s)")
    ap.add_argument("--serve-budget-gib", type=float, default=48.0, help="admission budget of the server")
    ap.add_argument("--serve-fig3", type=int, default=1,
                    help="also serve the Fig. 3 sequence (the rotation-light one is the default)")
    ap.add_argument("--serve-near", type=float, default=0.9,
                    help="second trace offered at this fraction of the measured capacity (0: skip)")
    args = ap.parse_args()
    AUTOTUNE[0] = bool(args.autotune)
    if args.case == "ntt":
        run_case_ntt(args)
    elif args.case == "ks":
        run_case_ks(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
