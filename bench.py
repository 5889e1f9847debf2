"""Benchmark: extrapolated blocks/s of batched Fast Selective Extrapolation.

Workload (one step = one pass of the whole hot path over one batch): the
512x512 synthetic image, 4096 concealment blocks of 32x32 with the centred
16x16 loss area, DCT u WHT dictionary (K = 2048), I = 100, gamma = 0.5,
rho_hat = 0.8.  Every step rebuilds the table C (Alg. 2), packs the
operands, computes the initial projections (eq. 12) and runs the iterations
(Alg. 3) through the C ABI.  L2 is flushed (256 MiB write) between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec bf16x6]

``--impl reference`` times the FP64 CPU oracle (Alg. 1) on the host cores on
a bounded sample of the same workload.  Under torchrun (N > 1) each rank
runs its own full batch (weak scaling, no collective on the data path);
rank 0 prints one JSON line.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "extrapolated blocks/s (32x32 area, K=2048, 100 iters)"
UNIT = "blocks/s"
WORKLOAD = "img512_4096blk_32x32_16x16loss_dctwht_K2048_I100_rho0.8_gamma0.5"
# Launch shapes of the iteration kernel by autotuner variant, and the
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the shape the
# traffic was captured for (ncu on this workload, see profiles/); None for a
# shape without a capture or once the kernel changes.
ITERATE_SHAPES = {0: "iterate_f32_kernel<1,64,4>", 1: "iterate_f32_kernel<2,32,1>"}
TRAFFIC_ITERATE = {0: 46.37e6}
SYM_SHAPES = {0: "iterate_sym_kernel<64>", 1: "iterate_sym_smem_kernel<64,3,9>", 2: "iterate_sym_tmem_kernel",
              3: "iterate_sym_hot_kernel<64,3,9>", 4: "iterate_sym_hot_kernel<64,3,9,1,2> with the model of eq. 9"}
TRAFFIC_ITERATE_SYM = {1: 36.91e6, 3: 36.92e6}
# On-chip roofs of the parity-class iteration kernel as ncu measured them per
# launch shape (fractions of peak; see profiles/).
ONCHIP_ITERATE_SYM = {
    1: {"l1tex_data_pipe_busy": 0.795, "l2_throughput": 0.338, "issue_active": 0.465,
        "source": "ncu --set full, profiles/iterate_sym_img512_4096blk.md"},
    3: {"l1tex_data_pipe_busy": 0.672, "l1tex_data_pipe_busy_of_active": 0.723, "l2_throughput": 0.365,
        "issue_active": 0.565, "source": "ncu --set full, profiles/iterate_sym_hot_img512_4096blk.md"},
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Weak scaling: every rank processes its own units; value = all units / job time."""
    return world * units_per_rank * steps / seconds


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def _oracle_setup(wl):
    import oracle as O
    phi = O.dict_dct_wht(wl.M, wl.N)
    return O, phi, O.find_duplicates(phi), O.weights(wl.M, wl.N, wl.rho_hat, wl.support)


def cpu_baseline(wl, n_blocks: int, threads: int = 0, margins: bool = False):
    """Time the FP64 oracle's original SE (Alg. 1) on the host cores over the
    first n_blocks blocks: (blocks/s, cores, seconds[, (out, u, c, margin)])."""
    O, phi, dup, w = _oracle_setup(wl)
    s = np.ascontiguousarray(wl.samples[:n_blocks])
    cores = threads if threads > 0 else O.max_threads()
    t0 = time.perf_counter()
    res = O.se_original_batch(phi, w, s, wl.gamma, wl.iterations, dup, nthreads=cores, margins=margins)
    dt = time.perf_counter() - t0
    assert res[-1] == 0
    if margins:
        return n_blocks / dt, cores, dt, res[:4]
    return n_blocks / dt, cores, dt


class FaseBaseline:
    """The oracle's fast form on the host cores: Alg. 2 (the tables, once per
    pattern, timed on its own) and Alg. 3 over the blocks (timed per batch)."""

    def __init__(self, wl, threads: int = 0):
        self.O, self.phi, self.dup, self.w = _oracle_setup(wl)
        self.wl = wl
        self.cores = threads if threads > 0 else self.O.max_threads()
        t0 = time.perf_counter()
        self.C, self.D = self.O.fase_tables(self.phi, self.w)
        self.tables_s = time.perf_counter() - t0

    def run(self, n_blocks: int):
        """Alg. 3 over the first n_blocks blocks; returns (blocks/s, seconds)."""
        s = np.ascontiguousarray(self.wl.samples[:n_blocks])
        t0 = time.perf_counter()
        _out, _u, _c, st = self.O.fase_batch(self.phi, self.w, self.C, self.D, s, self.wl.gamma,
                                             self.wl.iterations, self.dup, nthreads=self.cores)
        dt = time.perf_counter() - t0
        assert st == 0
        return n_blocks / dt, dt


def _psnr_sub(est, truth, loss):
    """PSNR pooled over the loss pixels of all blocks (10 log10(255^2 / MSE))."""
    d = est[:, loss] - truth[:, loss]
    return 10.0 * np.log10(255.0 ** 2 / float(np.mean(d * d)))


def calibrated_sample(wl, seconds: float) -> int:
    """Blocks of the oracle that take about `seconds` on the host cores (from a 16-block run)."""
    rate, _, _ = cpu_baseline(wl, 16)
    return int(max(16, min(wl.B, rate * seconds)))


def run_reference(args):
    """The reference arm: the oracle's fast form (Alg. 2 + 3, FP64 C) on all host
    cores, the fair CPU baseline; each step is the whole 4096-block batch
    through Alg. 3, the tables (Alg. 2) built once per pattern beforehand and
    listed separately."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2204_14194_gb300 import workloads as W
    wl = W.config2()
    nb = min(args.ref_sample or wl.B, wl.B)
    fb = FaseBaseline(wl)
    for _ in range(args.warmup):
        fb.run(max(1, nb // 8))
    secs = []
    for _ in range(args.steps):
        secs.append(fb.run(nb)[1])
    value = nb * args.steps / sum(secs)
    which = f"all {wl.B} blocks" if nb == wl.B else f"first {nb} of the {wl.B} blocks"
    sample = f"{which} per step, FaSE (Alg. 3) in fp64 C; tables (Alg. 2) built once, {fb.tables_s:.2f} s"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "blocks": wl.B, "blocks_per_step": nb, "form": "fase (Alg. 2 + 3)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": fb.cores, "kind": "oracle",
                         "sample": sample, "tables_s": fb.tables_s},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2204_14194_gb300 import binding as B
    from paper_2204_14194_gb300 import opcount
    from paper_2204_14194_gb300 import workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = W.config2()
    n, M, N, K, I = wl.B, wl.M, wl.N, wl.K, wl.iterations
    ctx = B.Context(local)
    plan = ctx.plan(M, N, wl.basis, K, wl.rho_hat, wl.gamma, I, prec=args.prec, products=args.products)
    # AUTO takes the transform-domain products for this separable dictionary
    products = "dense" if args.products == "dense" else "transform"
    stream = torch.cuda.Stream(device=dev)
    s_d = torch.from_numpy(wl.samples).to(dev)
    out_d = torch.empty_like(s_d)
    u_d = torch.empty((n, I), dtype=torch.int32, device=dev)
    c_d = torch.empty((n, I), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        plan.reset_tables()
        plan.extrapolate_strided(s_d, out_d, u_d, c_d, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    ctx.sync(stream)
    torch.cuda.synchronize()

    # ---- timed region: device time of exactly K steps, L2 flushed between them
    launches0 = ctx.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ctx.sync(stream)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    launches = ctx.stats()["kernel_launches"] - launches0
    total_ms = max_over_ranks(sum(step_ms))
    value = job_throughput(n, ws, args.steps, total_ms / 1000.0)

    # ---- sustained pass: the same step back to back for about --sustain-s
    # seconds (L2 flushed between steps), with its own clock record, so that
    # the clocks are sampled many times while the GPU is busy
    sustained = None
    if args.sustain_s > 0:
        sus_steps = max(1, int(args.sustain_s * 1000.0 / max(total_ms / args.steps + 0.05, 1e-3)))
        sus_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(sus_steps)]
        clocks_s = ClockSampler(local)
        clocks_s.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(sus_steps):
                flush.fill_(float(i))
                sus_ev[i][0].record(stream)
                step()
                sus_ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        clk_s = clocks_s.stop()
        ctx.sync(stream)
        sus_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in sus_ev))
        sustained = {"steps": sus_steps, "seconds_wall": wall, "value": job_throughput(n, ws, sus_steps, sus_ms / 1000.0),
                     "ms_per_step": sus_ms / sus_steps, "clocks": clk_s,
                     "timing": "CUDA events around each step; the L2 flush between steps is outside them"}

    # ---- the same steps with the table kept across steps (built once per pattern,
    # Sec. V: the paper times table generation apart from the per-block cost),
    # device time with CUDA events, L2 flushed between steps
    cached_steps = max(args.steps, 20)
    with torch.cuda.stream(stream):
        plan.extrapolate_strided(s_d, out_d, u_d, c_d, stream=stream)   # builds the table
        cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(cached_steps)]
        for i in range(cached_steps):
            flush.fill_(float(i))
            cev[i][0].record(stream)
            plan.extrapolate_strided(s_d, out_d, u_d, c_d, stream=stream)
            cev[i][1].record(stream)
    torch.cuda.synchronize()
    cached_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in cev))
    table_cached = {"value": job_throughput(n, ws, cached_steps, cached_ms / 1000.0), "unit": UNIT,
                    "ms_per_step": cached_ms / cached_steps, "steps": cached_steps,
                    "what": "the same step with the table of Alg. 2 built once before the steps and kept "
                            "(one pattern for every step), CUDA events per step, L2 flushed between steps"}

    # ---- per-stage device times (CUDA events around each stage on the launching
    # stream), in a separate pass so that the events do not touch the timed steps
    prof_steps = min(args.steps, 100)
    ctx.set_profiling(True)
    ctx.stage_times(reset=True)
    with torch.cuda.stream(stream):
        for i in range(prof_steps):
            flush.fill_(float(i))
            step()
    ctx.sync(stream)
    stages = ctx.stage_times(reset=True)
    # the same stages with the table kept (no table build beside the projections)
    with torch.cuda.stream(stream):
        plan.extrapolate_strided(s_d, out_d, u_d, c_d, stream=stream)
    ctx.sync(stream)
    ctx.stage_times(reset=True)
    with torch.cuda.stream(stream):
        for i in range(prof_steps):
            flush.fill_(float(i))
            plan.extrapolate_strided(s_d, out_d, u_d, c_d, stream=stream)
    ctx.sync(stream)
    stages_cached = ctx.stage_times(reset=True)
    ctx.set_profiling(False)

    # ---- end to end through the host-buffer entry point (pinned host memory):
    # in place (the caller's image buffer receives the loss areas; the kernels
    # read the support samples and write the loss areas over the host link),
    # and with a separate output buffer (every sample in, every result out)
    s_h = torch.from_numpy(wl.samples).pin_memory()
    o_h = torch.empty_like(s_h).pin_memory()
    ip_h = torch.from_numpy(wl.samples).pin_memory()

    e2e_steps = max(args.steps, 200)   # host wall clock: enough calls to average out host jitter

    def e2e_rate(src, dst):
        for _ in range(3):
            plan.extrapolate_host(src, dst)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.reset_tables()
            plan.extrapolate_host(src, dst)
        return job_throughput(n, ws, e2e_steps, max_over_ranks(time.perf_counter() - t0))

    e2e_sync = e2e_rate(ip_h, ip_h)
    e2e_separate = e2e_rate(s_h, o_h)
    ip_ok = bool(np.array_equal(ip_h.numpy(), o_h.numpy()))

    # the same steps through the asynchronous host-buffer call, three images in
    # flight (each step has its own pinned image buffer, extrapolated in place:
    # its samples are copied in and the rows of its loss box copied out by the
    # copy engines while the other steps compute); every ticket is waited for
    # inside the timed region
    ring = [torch.from_numpy(wl.samples).pin_memory() for _ in range(3)]

    def e2e_async_rate():
        for i in range(3):
            ctx.host_wait(plan.extrapolate_host_async(ring[i], ring[i]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pending = []
        for i in range(e2e_steps):
            if len(pending) == len(ring):
                ctx.host_wait(pending.pop(0))
            plan.reset_tables()
            buf = ring[i % len(ring)]
            pending.append(plan.extrapolate_host_async(buf, buf))
        for t in pending:
            ctx.host_wait(t)
        return job_throughput(n, ws, e2e_steps, max_over_ranks(time.perf_counter() - t0))

    e2e_value = e2e_async_rate()
    async_ok = all(bool(np.array_equal(b.numpy(), o_h.numpy())) for b in ring)
    rows, cols = np.nonzero(wl.support == 0)
    # samples copied out per block in place: from the first to the last sample of the loss box
    span = int((rows.max() - rows.min()) * N + cols.max() - cols.min() + 1) if len(rows) else 0

    # ---- error against the fp64 form, and the fp64 form's own throughput
    out_m, u_m, c_m = out_d.cpu().numpy(), u_d.cpu().numpy(), c_d.cpu().numpy()
    plan64 = ctx.plan(M, N, wl.basis, K, wl.rho_hat, wl.gamma, I, prec="fp64", products=args.products)
    o64 = torch.empty_like(s_d)
    u64 = torch.empty_like(u_d)
    c64 = torch.empty_like(c_d)
    plan64.extrapolate_strided(s_d, o64, u64, c64, stream=stream)
    ctx.sync(stream)
    fp64_steps = max(1, min(3, args.steps))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(fp64_steps):
            plan64.reset_tables()
            plan64.extrapolate_strided(s_d, o64, u64, c64, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    fp64_value = n * fp64_steps / (e0.elapsed_time(e1) / 1000.0)
    o64, u64, c64 = o64.cpu().numpy(), u64.cpu().numpy(), c64.cpu().numpy()
    same = np.all(u_m == u64, axis=1)
    first_diff = np.where(same, I, np.argmax(u_m != u64, axis=1))
    rel = []
    for b in range(n):
        t = first_diff[b]
        if t:
            ref = c64[b, :t]
            rel.append(np.max(np.abs(c_m[b, :t] - ref) / np.maximum(np.abs(ref), 1e-12 * np.max(np.abs(ref)))))
    loss = wl.support == 0
    gt = wl.samples[:, loss]

    def _psnr(o):
        d = o[:, loss] - gt
        return 10.0 * np.log10(255.0 ** 2 / float(np.mean(d * d)))

    # ---- roofline of the dominant kernel (the iteration kernel, Alg. 3).  Its
    # table stays in L2 and its projections on chip, so HBM does not bind it:
    # achieved = the kernel's own Table-I operations (scores, maximum,
    # coefficient, update: I*(5K/4 + 5) per block with parity classes) /
    # average launch time, against the fp32 CUDA-core rate (152 SMs x 128
    # lanes x 2 flops x max SM clock) as context; the binding roofs are the
    # on-chip data paths, whose busy fractions come from the ncu capture.
    hbm_peak, tc_peak, peak_kind = measured_peaks()
    it_ms, it_n = stages["iterate"]
    it_avg_s = it_ms / max(it_n, 1) / 1000.0
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    info = plan.info()
    variant = max(ctx.tuned_variant("iterate:f32:%d" % K), 0)
    if info.get("iterations") == "parity-classes":
        # the kernel's own work: scores, maximum, coefficient and update of one
        # class (a quarter of the atoms) per iteration; the model accumulate of
        # eq. (9) (2 flops per loss pixel and iteration) when the kernel
        # evaluates the model itself, else the model kernel does
        ops = n * I * opcount.fase_select_update_ops(M, N, K, classes=4)
        nb = 1 << max(n - 1, 0).bit_length()
        rows, cols = np.nonzero(wl.support == 0)
        mkey = "sym:f32:%d:n%d:model%dx%d" % (K, nb, rows.max() - rows.min() + 1, cols.max() - cols.min() + 1)
        sv = ctx.tuned_variant(mkey)
        if sv < 0:
            sv = max(ctx.tuned_variant("sym:f32:%d:n%d" % (K, nb)), 0)
        if sv == 4:
            ops += n * I * 2 * int(np.sum(wl.support == 0))
        it_kernel, it_traffic = SYM_SHAPES.get(sv, "iterate_sym kernel") + " (parity classes)", \
            TRAFFIC_ITERATE_SYM.get(sv)
        row_bytes = K // 4 * 4
    else:
        ops = n * I * opcount.fase_select_update_ops(M, N, K)
        row_bytes = K * 4
        if args.prec == "certified":   # one launch shape; the stage also holds the fp64 recomputation
            it_kernel, it_traffic = "iterate_f32_kernel<1,64,4> certified form + fp64 recomputation", None
        else:
            it_kernel, it_traffic = ITERATE_SHAPES.get(variant, "iterate_f32_kernel"), TRAFFIC_ITERATE.get(variant)
    achieved = ops / it_avg_s / 1e12
    roofline = {"kernel": it_kernel, "bound": "alu", "achieved": achieved,
                "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": it_traffic,
                "peak_kind": "derived: 152 SMs x 128 fp32 lanes x 2 flops x 2.07 GHz",
                "l2_read_GBps": n * (I - 1) * row_bytes / it_avg_s / 1e9, "plan": info}
    if info.get("iterations") == "parity-classes" and sv in ONCHIP_ITERATE_SYM:
        # the roofs the kernel meets on chip, as ncu measured them for this
        # launch shape (busy fraction of the L1/shared data pipe, L2 throughput)
        roofline["onchip"] = dict(ONCHIP_ITERATE_SYM[sv])
    pr_ms, pr_n = stages["projections"]
    pr_avg_s = pr_ms / max(pr_n, 1) / 1000.0
    na = int(np.sum(wl.support))
    if products == "transform":
        # eq. 12 as two separable 2-D transforms per block (DCT and WHT halves):
        # 2 MN (M + N) flops each; algorithmic bytes: samples on A read and
        # written to the output (8 B each), R^(0) written (4 B per atom)
        ntr = 2 if wl.basis == "dct_wht" else 1
        if args.prec == "fp64":
            roofline_gemm = None
        else:
            gbs = n * (16.0 * na + 4.0 * K) / pr_avg_s / 1e9
            if info.get("projections") == "split-tf32":
                # four folded quarter transforms per block as m16n8k8 tensor products in
                # split TF32 (3 products each): bound by the block's bytes, not its flops
                tflops = n * 3 * ntr * M * N * (M + N) / pr_avg_s / 1e12
                pc_ms, pc_n = stages_cached["projections"]
                gbs_c = n * (16.0 * na + 4.0 * K) / (pc_ms / max(pc_n, 1) / 1000.0) / 1e9 if pc_n else None
                roofline_gemm = {
                    "kernel": "sym_r0_32tc_kernel (eq. 12, folded quarter transforms, mma.sync split TF32)",
                    "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "tensor_tflops": tflops, "peak_kind": peak_kind + " HBM copy",
                    "bytes_per_block": "16 |A| (samples read, support copied to out) + 4 K (R0 written)",
                    "note": "the step rebuilds the table beside the projections, which share the SMs with it",
                    "table_kept": None if gbs_c is None else {
                        "achieved": gbs_c, "frac": gbs_c / hbm_peak,
                        "what": "the same kernel in steps that keep the table (nothing runs beside it)"}}
            else:
                if info.get("iterations") == "parity-classes":
                    # folded into four quarter-size transforms per block: half the flops
                    flops, pk = ntr * M * N * (M + N), \
                        "sym_r0_kernel<%d,%d> (eq. 12, four folded quarter transforms)" % (M // 2, N // 2)
                else:
                    flops, pk = ntr * 2.0 * M * N * (M + N), \
                        "sep_warp_kernel<32,32,8,4> (eq. 12 as separable transforms, Sec. VI)"
                tflops = n * flops / pr_avg_s / 1e12
                roofline_gemm = {
                    "kernel": pk,
                    "bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": tflops / alu_peak, "hbm_GBps": gbs, "hbm_frac": gbs / hbm_peak,
                    "peak_kind": "derived: 152 SMs x 128 fp32 lanes x 2 flops x 2.07 GHz"}
    else:
        npairs = {"bf16x6": 6, "bf16x3": 3, "bf16": 1}.get(args.prec, 0)
        tflops = 2.0 * K * n * na * npairs / pr_avg_s / 1e12 if npairs else None
        roofline_gemm = None if tflops is None else {
            "kernel": "tc_gemm_kernel<128,%d,1> (eq. 12 projections, every split part of a k-slice per stage)"
                      % {6: 3, 3: 2, 1: 1}.get(npairs, 3), "bound": "tensor",
            "achieved": tflops, "peak": tc_peak, "unit": "TFLOP/s", "frac": tflops / tc_peak,
            "peak_kind": peak_kind + " bf16 dense"}

    cpu = None
    vs_oracle = None
    if rank == 0 and not args.no_cpu_baseline:
        # original SE (Alg. 1) on a bounded sample, with its tie margins: the
        # parity of the measured outputs against the oracle on those blocks
        sample = args.ref_sample or calibrated_sample(wl, 15.0)
        v_se, cores, dt, (ro, ru, rc, rm) = cpu_baseline(wl, sample, margins=True)
        tie_free, errs, same_to_tie = 0, [], 0
        for b in range(sample):
            bad = np.nonzero(rm[b] <= 1e-4)[0]
            t = int(bad[0]) if len(bad) else I
            tie_free += t == I
            same_to_tie += bool(np.all(u_m[b, :t] == ru[b, :t]))
            if t:
                ref = rc[b, :t]
                errs.append(float(np.max(np.abs(c_m[b, :t] - ref) /
                                         np.maximum(np.abs(ref), 1e-12 * np.max(np.abs(ref))))))
        lm = wl.support == 0
        d_or = ro[:, lm] - wl.samples[:sample][:, lm]
        vs_oracle = {"blocks": sample, "tie_margin": 1e-4, "tie_free_frac": tie_free / sample,
                     "index_identical_to_first_near_tie_frac": same_to_tie / sample,
                     "max_rel_coef_err_to_first_near_tie": max(errs) if errs else 0.0,
                     "psnr_db": _psnr_sub(out_m[:sample], wl.samples[:sample], lm),
                     "psnr_oracle_db": 10.0 * np.log10(255.0 ** 2 / float(np.mean(d_or * d_or))),
                     "what": "the fp32 results of the timed steps against the FP64 oracle (Alg. 1) "
                             "on the first blocks of the batch"}
        # the fast form (Alg. 2 + 3) on all cores, the fair CPU baseline
        fb = FaseBaseline(wl)
        v_fase, fase_s = fb.run(n)
        cpu = {"value": v_fase, "unit": UNIT, "cores": fb.cores, "kind": "oracle",
               "sample": f"FaSE (Alg. 3, fp64 C) over all {n} blocks, {fase_s:.2f} s; tables (Alg. 2) "
                         f"once per pattern, {fb.tables_s:.2f} s, not counted; original SE (Alg. 1) "
                         f"over the first {sample} blocks, {dt:.1f} s",
               "value_fase": v_fase, "value_se": v_se, "tables_s": fb.tables_s}

    sorted_ms = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "blocks_per_gpu": n, "M": M, "N": N, "K": K,
                   "iterations": I, "products": products,
                   "precision": ("fp32 separable transforms for tables and projections" if products == "transform"
                                 else args.prec + " tensor-core products") + ", fp32 recurrence"
                                if args.prec != "fp64" else "fp64 throughout",
                   "certified": args.prec == "certified",
                   "tables": "rebuilt every step", "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(sorted_ms, 50)), "p99": float(np.percentile(sorted_ms, 99)),
                       "what": "per-batch (4096 blocks) device time"},
        "stages_ms_per_step": {k: v[0] / prof_steps for k, v in stages.items()},
        "stages_note": f"CUDA events around each stage, separate pass of {prof_steps} steps",
        "gpu_launches": int(launches),
        "clocks": clk,
        "table_cached": table_cached,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(n * M * N * 8),
                "d2h_bytes_per_step": int(n * span * 8),
                "how": "se_extrapolate_host_async in place on pinned host buffers, three steps in flight "
                       "(every sample copied in, of each block the span of its loss box copied out, by the "
                       "copy engines), host wall clock over %d steps, table rebuilt every step, every ticket "
                       "waited for inside the timed region" % e2e_steps,
                "results_equal_device_path": async_ok,
                "synchronous_calls": {
                    "value": e2e_sync, "h2d_bytes_per_step": int(n * int(np.sum(wl.support)) * 8),
                    "d2h_bytes_per_step": int(n * int(np.sum(wl.support == 0)) * 8),
                    "how": "se_extrapolate_host in place on pinned host buffers, one call at a time (support "
                           "samples in, loss areas out, read and written by the kernels over the host link)",
                    "in_place_equals_separate_buffers": ip_ok},
                "separate_buffers": {"value": e2e_separate, "h2d_bytes_per_step": int(n * M * N * 8),
                                     "d2h_bytes_per_step": int(n * M * N * 8),
                                     "how": "se_extrapolate_host, one call at a time"}},
        "roofline": roofline,
        "roofline_projections": roofline_gemm,
        "vs_fp64_form": {"fp64_blocks_per_s": fp64_value, "speedup": value / fp64_value,
                         "index_sequence_identical_frac": float(np.mean(same)),
                         "max_rel_coef_err_before_first_divergence": float(max(rel)) if rel else 0.0,
                         "psnr_db": _psnr(out_m), "psnr_fp64_db": _psnr(o64)},
        "vs_oracle": vs_oracle,
        "cpu_baseline": cpu,
    }
    if sustained is not None:
        line["sustained"] = sustained
    if rank == 0 and args.secondary and args.prec != "fp64":
        # secondary measurements recorded in the same line: the Gaussian-dictionary
        # workload, the mixed-size batch and a short serving run at the mixed-size
        # request stream
        line["gauss1080"] = secondary_gauss1080(args.prec)
        # the mixed-size batch with per-block masks (20000 blocks of 16, 32 and 64
        # samples square, I from 50 to 500): lazy columns, one stream per size
        line["mixed"] = measure_workload("mixed", 0, 3, 3, args.prec)
        line["serving"] = [serve_measure(float(r), args.serve_s, 0.5, args.gauss_share, args.budget_gb, args.prec)
                           for r in args.serve_rates.split(",")]
    if args.prec == "certified":
        cs = ctx.cert_stats()
        line["certified"] = {"blocks": cs["blocks"], "recomputed_in_fp64": cs["recomputed"],
                             "recomputed_frac": cs["recomputed"] / max(cs["blocks"], 1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan64.close()
    plan.close()
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_workload(args):
    """Secondary measurements (not the headline): the 1920x1080 Gaussian-dictionary
    workload (shared pattern, K = 4096, I = 200) and the mixed-size workload with
    per-block masks (16/32/64 areas, I in [50, 500])."""
    print(json.dumps(measure_workload(args.workload, args.blocks, args.steps, args.warmup, args.prec,
                                      args.no_graphs)), flush=True)
    return 0


def measure_workload(workload: str, blocks: int, steps: int, warmup: int, prec: str, no_graphs: bool = False):
    """One secondary workload's line (see run_workload)."""
    import torch
    from paper_2204_14194_gb300 import binding as B
    from paper_2204_14194_gb300 import workloads as W

    # one context (and stream) per plan, so the three area sizes overlap on the device
    ctxs, streams, groups = [], [], []
    if workload in ("dft64", "video"):
        # complex DFT atoms on 64 x 64 areas (the processing-time scenario of the
        # paper's Fig. 7: K = 4096, 32 x 32 loss) or 3-D video blocks 16 x 16 x 4
        # with 3-D DCT atoms (K = 1024); I = 100, gamma = 0.5, rho_hat = 0.8
        ctxs.append(B.Context(0))
        streams.append(torch.cuda.Stream())
        if workload == "dft64":
            n = blocks or 1024
            plan = ctxs[0].plan(64, 64, "dft", 4096, 0.8, 0.5, 100, prec=prec)
            samples = W.tiled_image(2048, 2048, 64)
            rng = np.random.default_rng(64)
            corners = rng.integers(0, 2048 - 64, size=(n, 2))
            samples = np.stack([samples[r:r + 64, c:c + 64] for r, c in corners])
            name = "dft_64x64_K4096_I100_%dblk" % n
        else:
            n = blocks or 4096
            plan = ctxs[0].plan(16, 16, "dct", 1024, 0.8, 0.5, 100, prec=prec, T=4)
            samples = np.stack([W.video_block(16, 16, 4, 20000 + i) for i in range(n)])
            name = "video_16x16x4_dct_K1024_I100_%dblk" % n
        s = torch.from_numpy(np.ascontiguousarray(samples)).cuda()
        groups.append((plan, s, torch.empty_like(s), None, 100))
    elif workload == "gauss1080":
        wl = W.config3(blocks or None)
        ctxs.append(B.Context(0))
        streams.append(torch.cuda.Stream())
        plan = ctxs[0].plan(32, 32, "numeric", 4096, wl.rho_hat, wl.gamma, wl.iterations, prec=prec,
                            dictionary=wl.dictionary)
        s = torch.from_numpy(wl.samples).cuda()
        groups.append((plan, s, torch.empty_like(s), None, wl.iterations))
        name = wl.name
    else:
        for wl in W.config4(blocks or 20000):
            c = B.Context(0)
            ctxs.append(c)
            streams.append(torch.cuda.Stream())
            plan = c.plan(wl.M, wl.N, "dct_wht", wl.K, wl.rho_hat, wl.gamma, int(wl.iters_per_block.max()),
                          prec=prec)
            s = torch.from_numpy(wl.samples).cuda()
            m = torch.from_numpy(wl.support).cuda()
            groups.append((plan, s, torch.empty_like(s), m, wl.iters_per_block))
        name = "mixed_%dblk_16-32-64_masks_I50-500" % sum(g[1].shape[0] for g in groups)
    descs = [None if g[3] is None else
             [{"samples": g[1][b], "support": g[3][b], "out": g[2][b], "iterations": int(g[4][b])}
              for b in range(g[1].shape[0])] for g in groups]

    for c in ctxs:
        c.set_graphs(not no_graphs)

    def step():
        for (plan, s, o, m, it), d, stream in zip(groups, descs, streams):
            plan.reset_tables()
            if d is None:
                plan.extrapolate_strided(s, o, stream=stream)
            else:
                plan.extrapolate_batch(d, stream=stream)

    def sync():
        for c, st in zip(ctxs, streams):
            c.sync(st)

    for _ in range(warmup):
        step()
    sync()
    for c in ctxs:
        c.set_profiling(True)
        c.stage_times(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    sync()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0 / steps
    nb = sum(g[1].shape[0] for g in groups)
    stages = {}
    for c in ctxs:
        for k, v in c.stage_times(reset=True).items():
            stages[k] = stages.get(k, 0.0) + v[0] / steps
    line = {"metric": "extrapolated blocks/s", "workload": name, "value": nb / (ms / 1000.0),
            "unit": "blocks/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "precision": prec, "timing": "host wall clock around the steps (several streams)",
            "graphs": not no_graphs,
            "tuning": [c.tuning_stats() for c in ctxs],
            "stages_ms_per_step_summed_over_streams": stages}
    for c in ctxs:
        c.close()
    return line


def run_single(args):
    """Latency of one 32 x 32 block (the single-block workload: one patch, K = 2048
    DCT u WHT, I = 100): device time per call with CUDA events, table cached and
    rebuilt before every call, in the default (fp32) and the fp64 form."""
    import torch
    from paper_2204_14194_gb300 import binding as B
    from paper_2204_14194_gb300 import workloads as W

    wl = W.config1()
    ctx = B.Context(0)
    stream = torch.cuda.Stream()
    s = torch.from_numpy(wl.samples).cuda()
    out = torch.empty_like(s)
    res = {}
    for prec in ("bf16x6", "fp64"):
        plan = ctx.plan(32, 32, wl.basis, wl.K, wl.rho_hat, wl.gamma, wl.iterations, prec=prec,
                        products=args.products)
        for rebuild in (False, True):
            for _ in range(max(args.warmup, 3)):
                plan.extrapolate_strided(s, out, stream=stream)
            ctx.sync(stream)
            ms = []
            for _ in range(args.steps):
                if rebuild:
                    plan.reset_tables()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a.record(stream)
                    plan.extrapolate_strided(s, out, stream=stream)
                    b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            res[f"{prec}_{'tables_rebuilt' if rebuild else 'tables_cached'}"] = {
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99))}
        plan.close()
    print(json.dumps({"metric": "single-block latency (32x32 area, K=2048, 100 iters)", "unit": "ms",
                      "steps": args.steps, "latency": res,
                      "timing": "CUDA events around each call on its stream, synchronised per call"}), flush=True)
    ctx.close()
    return 0


def serve_measure(rate: float, duration: float, warm_s: float, gauss_share: float, budget_gb: float,
                  prec: str = "bf16x6"):
    """Serving measurement: open-loop Poisson arrivals of single-block requests of
    mixed area size (16/32/64), DCT u WHT or Gaussian dictionaries with K = 2MN,
    random per-request masks, I in [100, 300], under an HBM budget; latency is
    completion minus the scheduled arrival time.  Returns the result as a dict."""
    import threading as th
    from paper_2204_14194_gb300 import binding as B
    from paper_2204_14194_gb300 import workloads as W

    rng = np.random.default_rng(5)
    ctx = B.Context(0, hbm_budget_bytes=int(budget_gb * (1 << 30)))
    plans = {}
    for L in (16, 32, 64):
        plans[("dct_wht", L)] = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, 300, prec=prec)
        if gauss_share > 0:
            plans[("gauss", L)] = ctx.plan(L, L, "numeric", 2 * L * L, 0.8, 0.5, 300, prec=prec,
                                           dictionary=W.gaussian_dictionary(2 * L * L, L, L, 900 + L))
    pool = 256
    samp = {L: [W.patch(L, 50000 + 1000 * L + i) for i in range(pool)] for L in (16, 32, 64)}
    mrng = np.random.default_rng(6)
    masks = {L: [W.rect_support(L, L, mrng) if i % 2 else W.holes_support(L, L, mrng) for i in range(pool)]
             for L in (16, 32, 64)}
    # every plan is ready before the clock starts: one masked request each
    # prepares the plan's lazy-column operands and the tuner's choices
    for (kind, L), p in plans.items():
        o = np.empty((L, L))
        ctx.poll(ctx.submit(p, samp[L][0], o, iterations=300, support=masks[L][0]), timeout_us=-1)
    total_t = warm_s + duration
    n = int(rate * total_t)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sizes = rng.choice([16, 32, 64], size=n)
    gauss = rng.random(n) < gauss_share
    iters = rng.integers(100, 301, size=n)
    pick = rng.integers(0, pool, size=n)
    outs = {L: np.empty((pool, L, L)) for L in (16, 32, 64)}   # results are not checked here
    tickets = [None] * n
    t_sub = np.zeros(n)
    lat = np.full(n, np.nan)
    start = time.perf_counter() + 0.2

    def submitter():
        for i in range(n):
            target = start + arrivals[i]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 2e-4:
                    time.sleep(target - now - 1e-4)
            L = int(sizes[i])
            p = plans[("gauss" if gauss[i] else "dct_wht", L)]
            t_sub[i] = time.perf_counter()
            tickets[i] = ctx.submit(p, samp[L][pick[i]], outs[L][pick[i]], iterations=int(iters[i]),
                                    support=masks[L][pick[i]])

    th_sub = th.Thread(target=submitter)
    th_sub.start()
    done = 0
    for i in range(n):
        while tickets[i] is None:
            time.sleep(1e-4)
        st, l = ctx.poll(tickets[i], timeout_us=-1)
        lat[i] = (t_sub[i] - (start + arrivals[i])) + l
        done += 1
    th_sub.join()
    t_end = time.perf_counter()
    keep = arrivals >= warm_s
    L_ms = lat[keep] * 1000.0
    thr = done / (t_end - start)
    res = {"workload": "poisson %.0f req/s, %.1f s (+%.1f s warm-up), areas 16/32/64, K = 2MN, %d%% Gaussian, "
                       "per-request masks, I in [100,300], budget %.0f GB" % (rate, duration, warm_s,
                                                                             100 * gauss_share, budget_gb),
           "offered_rate": rate, "requests": int(keep.sum()),
           "throughput_blocks_per_s": thr,
           "latency_ms": {"p50": float(np.percentile(L_ms, 50)), "p99": float(np.percentile(L_ms, 99)),
                          "max": float(L_ms.max())},
           "sustained": bool(thr >= 0.97 * rate),
           "serving_slices": ctx.stats()["serving_slices"], "precision": prec}
    ctx.close()
    return res


def run_serve(args):
    """The serving measurement alone (--workload serve)."""
    res = serve_measure(args.rate, args.duration, args.warm_s, args.gauss_share, args.budget_gb, args.prec)
    print(json.dumps({"metric": "serving latency and throughput", **res}), flush=True)
    return 0


def secondary_gauss1080(prec: str, steps: int = 5, warmup: int = 3, oracle_blocks: int = 24):
    """The 1920x1080 Gaussian-dictionary workload (8160 blocks of 32 x 32, K = 4096
    seeded Gaussian atoms, I = 200) as a secondary measurement: device-timed
    blocks/s with the table rebuilt every step and L2 flushed between steps,
    tensor-core throughput of the two product stages (split-bf16 products, six
    per product), and the error against the FP64 oracle (Alg. 1) on the first
    blocks."""
    import torch
    from paper_2204_14194_gb300 import binding as B
    from paper_2204_14194_gb300 import workloads as W

    wl = W.config3()
    n, I, K = wl.B, wl.iterations, 4096
    ctx = B.Context(0)
    stream = torch.cuda.Stream()
    plan = ctx.plan(32, 32, "numeric", K, wl.rho_hat, wl.gamma, I, prec=prec, dictionary=wl.dictionary)
    s_d = torch.from_numpy(wl.samples).cuda()
    out = torch.empty_like(s_d)
    u = torch.empty((n, I), dtype=torch.int32, device="cuda")
    c = torch.empty((n, I), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        plan.reset_tables()
        plan.extrapolate_strided(s_d, out, u, c, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.fill_(1.0)
            step()
    ctx.sync(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
    ctx.sync(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    ctx.set_profiling(True)
    ctx.stage_times(reset=True)
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))
            step()
    ctx.sync(stream)
    stages = {k: v[0] / steps for k, v in ctx.stage_times(reset=True).items()}
    ctx.set_profiling(False)
    o_m, u_m, c_m = out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()
    na = int(np.sum(wl.support))
    _hbm, tc_peak, peak_kind = measured_peaks()
    npairs = {"bf16x6": 6, "bf16x3": 3, "bf16": 1}.get(prec, 0)
    # the table of eq. 16 from two-part fp16 splits takes three products (fp16 runs at
    # the bf16 rate on the tensor cores)
    tpairs = 3 if plan.info().get("table_products") == "f16x3" else npairs
    tensor = None
    if npairs and stages.get("projections", 0) > 0 and stages.get("tables", 0) > 0:
        proj = 2.0 * K * n * na * npairs / (stages["projections"] / 1e3) / 1e12
        tab = 1.0 * K * (K + 1) * na * tpairs / (stages["tables"] / 1e3) / 1e12
        tensor = {"projections_tflops": proj, "tables_tflops": tab, "peak": tc_peak,
                  "projections_frac": proj / tc_peak, "tables_frac": tab / tc_peak,
                  "tables_ms": stages["tables"], "projections_ms": stages["projections"],
                  "peak_kind": peak_kind + " bf16 dense",
                  "flops": "split products counted: 2 K |A| n x %d (eq. 12), K (K + 1) |A| x %d "
                           "(eq. 16, the symmetric half)" % (npairs, tpairs)}
    # error against the FP64 oracle on the first blocks
    import oracle as O
    phi = np.ascontiguousarray(wl.dictionary, dtype=np.float64)
    dup = O.find_duplicates(phi)
    w = O.weights(32, 32, wl.rho_hat, wl.support)
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, np.ascontiguousarray(wl.samples[:oracle_blocks]),
                                             wl.gamma, I, dup, margins=True)
    assert st == 0
    tie_free, errs, same = 0, [], 0
    for b in range(oracle_blocks):
        bad = np.nonzero(rm[b] <= 1e-4)[0]
        t = int(bad[0]) if len(bad) else I
        tie_free += t == I
        same += bool(np.all(u_m[b, :t] == ru[b, :t]))
        if t:
            ref = rc[b, :t]
            errs.append(float(np.max(np.abs(c_m[b, :t] - ref) /
                                     np.maximum(np.abs(ref), 1e-12 * np.max(np.abs(ref))))))
    pm = wl.psnr_mask
    d_g = (o_m[:oracle_blocks] - wl.samples[:oracle_blocks])[pm[:oracle_blocks]]
    d_o = (ro - wl.samples[:oracle_blocks])[pm[:oracle_blocks]]
    res = {"workload": wl.name, "blocks": n, "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "precision": prec, "stages_ms_per_step": stages, "tensor": tensor,
           "vs_oracle": {"blocks": oracle_blocks, "tie_margin": 1e-4, "tie_free_frac": tie_free / oracle_blocks,
                         "index_identical_to_first_near_tie_frac": same / oracle_blocks,
                         "max_rel_coef_err_to_first_near_tie": max(errs) if errs else 0.0,
                         "psnr_db": 10.0 * np.log10(255.0 ** 2 / float(np.mean(d_g * d_g))),
                         "psnr_oracle_db": 10.0 * np.log10(255.0 ** 2 / float(np.mean(d_o * d_o)))},
           "timing": "CUDA events per step, table rebuilt every step, L2 flushed between steps"}
    plan.close()
    ctx.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "bf16", "fp64", "certified"])
    ap.add_argument("--products", default="auto", choices=["auto", "dense", "transform"],
                    help="scalar products of tables and projections (Sec. VI transforms or matrix products)")
    ap.add_argument("--no-graphs", action="store_true", help="launch the lazy rounds without CUDA graphs")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="oracle blocks per CPU measurement (0: sized from a calibration run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sustain-s", type=float, default=1.5,
                    help="seconds of the sustained pass after the timed steps (0: none)")
    ap.add_argument("--rate", type=float, default=50000.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: measured seconds")
    ap.add_argument("--serve-rates", default="50000,45000",
                    help="offered rates of the serving runs inside the headline run (its 'serving' key)")
    ap.add_argument("--serve-s", type=float, default=3.0,
                    help="serving seconds measured inside the headline run (its 'serving' key)")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the Gaussian-dictionary, mixed-batch and serving measurements of the headline run")
    ap.add_argument("--warm-s", type=float, default=1.0, help="serving: warm-up seconds")
    ap.add_argument("--gauss-share", type=float, default=0.5, help="serving: share of Gaussian dictionaries")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serving: HBM budget")
    ap.add_argument("--workload", default="img512",
                    choices=["img512", "gauss1080", "mixed", "serve", "single", "dft64", "video"],
                    help="img512 is the headline; the others are secondary measurements")
    ap.add_argument("--blocks", type=int, default=0, help="block count for --workload gauss1080/mixed")
    args = ap.parse_args()
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload != "img512":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
