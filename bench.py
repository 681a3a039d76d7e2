"""Benchmark: BF16 Stream-K GEMM shape sweep on GB300.

One step = one pass of the hot path over the five BF16 sweep problems
(3840x4096x4096, 1536x1536x8192, 8192x8192x8192, 2048x7168x1024,
128x8192x16384; BF16 inputs uniform[-1,1], FP32 accumulate, BF16 output),
each GEMM launched once in the library's default (Stream-K hybrid) mode.
Inputs are resident in HBM; before every GEMM a 256 MB buffer (twice L2) is
written and then read back, so the GEMM starts with none of its operands in
L2 and no dirty lines to write back; only the GEMMs are inside the
CUDA-event pairs.  The data-parallel
tiling baseline (same kernel, one whole tile per CTA per wave) is timed the
same way and reported beside it.

Prints ONE JSON line (rank 0).  Under torchrun every rank runs the full
workload on its own GPU (independent replicas, no collective on the data
path); value = total flops of all ranks / max over ranks of the time.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import workloads  # noqa: E402

METRIC = "GEMM TFLOP/s and % of dense peak, Stream-K vs data-parallel tiling, same GB300"
UNIT = "TFLOP/s"
WORKLOAD = ("BF16 Stream-K GEMM sweep (M,N,K) = " +
            " ".join(f"({m},{n},{k})" for m, n, k in workloads.BF16_SWEEP) +
            "; A row-major, B column-major, uniform[-1,1] -> BF16, FP32 accumulate, BF16 output")
L2_FLUSH_BYTES = 256 << 20
DOMINANT_SHAPE = (8192, 8192, 8192)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "sk_tc_kernel_bf16_8192cube.md")


# --------------------------------------------------------------------- util
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"bf16": float(p["bf16_tflops"]), "bf16_sustained": float(p["bf16_tflops_sustained"]),
                "hbm": float(p["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "fallback"}


KERNEL_SOURCES = ("common.cuh", "gemm_tc.cuh", "ptx.cuh", "sched.cuh")


def kernel_sources_digest() -> str:
    """Hash of the device code of the tcgen05 GEMM kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_00044_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel sources changed since the capture."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    mh = re.search(r"kernel_sources_digest:\s*([0-9a-f]+)", txt)
    mt = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mt or mh.group(1) != kernel_sources_digest():
        return None
    return float(mt.group(1))


class ClockSampler:
    """nvidia-smi clock/throttle sampling in the background (every 20 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        ident = str(gpu_index)
        try:   # nvidia-smi ignores CUDA_VISIBLE_DEVICES: address the GPU by UUID
            uuid = str(torch.cuda.get_device_properties(gpu_index).uuid)
            ident = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={ident}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


SLOWDOWN_REASONS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


def bad_clocks(c) -> bool:
    """A clock record the timing rules reject: a hardware or thermal
    slowdown reason, or an SM clock well below its maximum under load."""
    if not c:
        return False
    return bool(SLOWDOWN_REASONS & set(c.get("reasons", []))) or c["sm_mhz"] < 0.8 * c["sm_max_mhz"]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(work: float, seconds: float, world: int):
    """(total work over ranks, max time over ranks)."""
    if world <= 1:
        return work, seconds
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    t = torch.tensor([work, seconds], dtype=torch.float64, device=dev)
    w = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(w.item()), float(s.item())


# ------------------------------------------------------------ our GPU arm
def run_ours(args, world, rank, local):
    import paper_2407_00044_gb300 as sk

    dev = torch.device("cuda", torch.cuda.current_device())
    pk = peaks()
    shapes = list(workloads.BF16_SWEEP)
    if args.only:
        shapes = [tuple(int(x) for x in args.only.split(","))]
    data = []
    for i, (M, N, K) in enumerate(shapes):
        a = workloads.device_uniform((M, K), seed=1000 + 2 * i, device=dev)
        b = workloads.device_uniform((N, K), seed=1001 + 2 * i, device=dev).t()   # column-major
        c = torch.empty(M, N, dtype=torch.bfloat16, device=dev)
        data.append((a, b, c))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)
    ws = sk.default_workspace(dev)
    stream = torch.cuda.current_stream()

    def l2_flush(i):
        # Write a buffer twice the size of L2 (evicts every operand), then
        # read it back: the dirty lines are written back here, outside the
        # timed events, and L2 is left holding clean, unrelated lines.
        flush.fill_(float(i))
        torch.sum(flush, dim=0, out=flush_sink)

    def one_pass(cfg, evs=None):
        for i, (a, b, c) in enumerate(data):
            l2_flush(i)
            if evs is not None:
                evs[i][0].record(stream)
            sk.gemm(a, b, c, config=cfg, workspace=ws)
            if evs is not None:
                evs[i][1].record(stream)

    def timed(cfg, steps):
        evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in shapes] for _ in range(steps)]
        for s in range(steps):
            one_pass(cfg, evs[s])
        torch.cuda.synchronize()
        per_shape = [[evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(steps)] for i in range(len(shapes))]
        return per_shape

    # (--fixup / --num-ctas / --tile pin the Stream-K arm's protocol and plan,
    # e.g. to profile one fixup; by default the library chooses)
    tm, tn = (int(x) for x in args.tile.split("x")) if args.tile else (0, 0)
    auto = sk.Config(mode=args.mode, fixup=args.fixup, num_ctas=args.num_ctas, tile_m=tm, tile_n=tn)
    dp = sk.Config(mode="dp")
    for _ in range(args.warmup):
        one_pass(auto)
        if args.dp:
            one_pass(dp)
    torch.cuda.synchronize()
    if ws.status() != 0:
        raise RuntimeError("device status after warm-up")

    # ---- timed regions: the Stream-K (library default) arm, then the
    # data-parallel arm, each with its own clock record; if either record
    # shows a slowdown reason or a stuck clock, both arms are measured once
    # more (the first records are kept in the line).
    def timed_region(cfg):
        clocks = ClockSampler(local) if rank == 0 else None
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms = timed(cfg, args.steps)
        torch.cuda.synchronize()
        barrier(world)
        return ms, time.perf_counter() - t0, (clocks.stop() if clocks else None)

    def both_arms():
        sk_r = timed_region(auto)
        dp_r = timed_region(dp) if args.dp else sk_r
        return sk_r, dp_r

    (sk_ms, wall, clk), (dp_ms, dp_wall, dp_clk) = both_arms()
    first_clocks = None
    if world == 1 and (bad_clocks(clk) or bad_clocks(dp_clk)):
        first_clocks = {"sk": clk, "dp": dp_clk}
        (sk_ms, wall, clk), (dp_ms, dp_wall, dp_clk) = both_arms()
    if ws.status() != 0:
        raise RuntimeError("device status after timing")

    flops = [workloads.gemm_flops(*s) for s in shapes]
    step_ms = sum(statistics.mean(v) for v in sk_ms)
    total_flops_local = sum(flops) * args.steps
    total_flops, max_s = aggregate(total_flops_local, step_ms * args.steps / 1e3, world)
    value = total_flops / max_s / 1e12

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clk["sm_mhz"] if clk else 2070.0
    hw_at_clock = hw_dense_bf16(sms, clk_mhz)
    hw_at_max = hw_dense_bf16(sms, clk["sm_max_mhz"] if clk else 2070.0)
    per_shape = []
    for (M, N, K), f, t_sk, t_dp, (a, b, c) in zip(shapes, flops, sk_ms, dp_ms, data):
        ms_sk = statistics.median(t_sk)
        ms_dp = statistics.median(t_dp)
        info = sk.plan(sk.make_problem(a, b, c), auto)
        per_shape.append({
            "M": M, "N": N, "K": K,
            "tile": f"{info.tile_m}x{info.tile_n}", "mode": ["auto", "dp", "sk", "hybrid1", "hybrid2"][info.mode],
            "units": info.num_ctas, "fixup": ["owner", "last_arriver", "split", "split_cluster"][info.fixup],
            "ms": round(ms_sk, 4), "tflops": round(f / ms_sk / 1e9, 1),
            "pct_peak": round(100 * f / ms_sk / 1e9 / pk["bf16"], 1),
            "pct_hw": round(100 * f / ms_sk / 1e9 / hw_at_clock, 1),
            "dp_ms": round(ms_dp, 4), "dp_tflops": round(f / ms_dp / 1e9, 1),
            "sk_over_dp": round(ms_dp / ms_sk, 3),
        })
    dp_step_ms = sum(statistics.mean(v) for v in dp_ms)

    # ---- best fixed-tile configurations: every candidate (tile x stages x
    # mode) timed on this GPU; the best DP one is the data-parallel baseline
    # a hand-tuned fixed-tile kernel would reach, the best SK one bounds what
    # the library's own choice leaves on the table.
    best_dp_ms, best_sk_ms = [], []
    if args.search:
        for entry, (a, b, c) in zip(per_shape, data):
            res = []
            for cfg, _pred in sk.autotune.candidates(sk.make_problem(a, b, c)):
                for _ in range(2):
                    sk.gemm(a, b, c, config=cfg, workspace=ws)
                ms = _timed_region(lambda: sk.gemm(a, b, c, config=cfg, workspace=ws), args.search_steps,
                                   lambda: l2_flush(0))
                res.append((cfg, ms))
            f = workloads.gemm_flops(entry["M"], entry["N"], entry["K"])
            for key, sel, acc in (("best_dp", lambda m: m == "dp", best_dp_ms),
                                  ("best_sk", lambda m: m != "dp", best_sk_ms)):
                cfg, ms = min((r for r in res if sel(r[0].mode)), key=lambda r: r[1])
                acc.append(ms)
                entry[key] = {"tile": f"{cfg.tile_m}x{cfg.tile_n}", "stages": cfg.stages, "mode": cfg.mode,
                              "ms": round(ms, 4), "tflops": round(f / ms / 1e9, 1)}
            entry["candidates_timed"] = len(res)
        if ws.status() != 0:
            raise RuntimeError("device status after the candidate search")

    # roofline of the dominant launch (the 8192^3 GEMM)
    di = shapes.index(DOMINANT_SHAPE) if DOMINANT_SHAPE in shapes else 0
    dom_ms = statistics.mean(sk_ms[di])
    achieved = flops[di] / (dom_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": round(achieved, 1), "peak": pk["bf16"], "unit": "TFLOP/s",
                "frac": round(achieved / pk["bf16"], 4),
                # the committed capture is of the 8192^3 launch
                "traffic": profiled_traffic() if shapes[di] == DOMINANT_SHAPE else None,
                "kernel": "sk_tc_kernel<bf16,bf16,%s tile> on %dx%dx%d" % ((per_shape[di]["tile"],) + shapes[di]),
                "peak_source": f"{pk['source']} bf16 burst (the launch is timed alone)",
                # context: the same against the seconds-long sustained figure
                "frac_of_sustained": round(achieved / pk["bf16_sustained"], 4),
                # and against the tensor cores' own dense rate at the sampled
                # SM clock and at the maximum clock
                "frac_of_hw_dense_at_sampled_clock": round(achieved / hw_at_clock, 4),
                "frac_of_hw_dense_at_max_clock": round(achieved / hw_at_max, 4)}

    # ---- end-to-end through the public API with host buffers
    e2e = run_e2e(sk, shapes, data, args, ws, world) if args.e2e else None

    # ---- the other configurations (FP32, FP8, grouped, autograd), each
    # against its own data-parallel arm; not part of `value`
    configs = None
    if args.configs and not args.only:
        del data
        torch.cuda.empty_cache()
        steps_cfg = max(5, min(args.steps, 20))
        configs = {}
        for name in ("f32", "fp8", "grouped", "autograd"):
            configs[name] = workload_record(name, sk, dev, pk, steps_cfg, max(3, args.warmup),
                                            lambda: l2_flush(0))
            torch.cuda.empty_cache()

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic: seeded uniform[-1,1] rounded to BF16 (torch CUDA generator)",
        "config": {"workload": WORKLOAD,
                   "mode": "library default: tile and DP/SK split chosen by the runtime model (per shape below)",
                   "l2": "flushed before every GEMM by writing then reading a 256 MB buffer (outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "dp_baseline": {"value": round(sum(flops) / (dp_step_ms / 1e3) / 1e12, 2), "unit": UNIT,
                        "ms_per_step": round(dp_step_ms, 4), "clocks": dp_clk,
                        "wall_s_timed_region": round(dp_wall, 3)},
        "hw_dense_bf16": {"flop_per_clk_per_sm": SM_BF16_FLOP_PER_CLK, "sms": sms,
                          "at_sampled_clock": round(hw_at_clock, 1), "at_max_clock": round(hw_at_max, 1),
                          "unit": UNIT,
                          "note": "pct_peak uses the measured cuBLAS burst; pct_hw this rate at the sampled clock"},
        "shapes": per_shape,
        "best_fixed_tile": None if not best_dp_ms else {
            "dp": {"value": round(sum(flops) / (sum(best_dp_ms) / 1e3) / 1e12, 2), "unit": UNIT},
            "sk": {"value": round(sum(flops) / (sum(best_sk_ms) / 1e3) / 1e12, 2), "unit": UNIT},
            "protocol": f"every tile x stages x mode candidate, median of {args.search_steps} runs, L2 flushed"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": len(shapes) * args.steps,
        "clocks": clk,
        "wall_s_timed_region": round(wall, 3),
    }
    if configs is not None:
        line["configs"] = configs
    if first_clocks is not None:
        line["remeasured"] = {"first_clocks": first_clocks, "arms": "both arms measured again",
                              "why": "slowdown reason or SM clock below 80 % of its maximum"}
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    return line


def run_e2e(sk, shapes, data, args, ws, world):
    """Same metric through the public API with pinned HOST buffers: every
    step uploads A and B, runs the GEMMs and downloads C, all inside the
    timed events.  ``HostGemmPipeline`` overlaps problem i's GEMM with the
    next problem's upload and the previous one's download (three streams)."""
    host = []
    for (a, b, c) in data:
        ha = torch.empty(a.shape, dtype=a.dtype, pin_memory=True).copy_(a)
        hbt = torch.empty(b.t().shape, dtype=b.dtype, pin_memory=True).copy_(b.t())
        hc = torch.empty(c.shape, dtype=c.dtype, pin_memory=True)
        host.append((ha, hbt.t(), hc))
    pipe = sk.HostGemmPipeline(host, device=data[0][0].device, workspace=ws)
    stream = torch.cuda.current_stream()
    steps = max(1, args.steps)
    for _ in range(2):
        pipe.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pipe.run(join=False)   # consecutive steps overlap (each step's own copies stay inside it)
    pipe.join()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    flops = sum(workloads.gemm_flops(*s) for s in shapes)
    tot, mx = aggregate(flops * steps, ms * steps / 1e3, world)
    return {"value": round(tot / mx / 1e12, 2), "unit": UNIT, "h2d_bytes_per_step": int(pipe.bytes_in),
            "d2h_bytes_per_step": int(pipe.bytes_out), "ms_per_step": round(ms, 3),
            "overlap": "uploads, GEMMs and downloads on three streams (HostGemmPipeline); consecutive steps overlap"}


# ------------------------------------------------- other workloads (info)
def _timed_region(fn, steps, flush):
    """Median ms of fn() over `steps` runs, L2 flushed before each."""
    stream = torch.cuda.current_stream()
    evs = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs)


SM_BF16_FLOP_PER_CLK = 8192   # dense BF16 tcgen05 rate of one SM (M128 N256 K16 per 128 cycles)


def hw_dense_bf16(sms: int, mhz: float) -> float:
    """Dense BF16 tensor rate in TFLOP/s of `sms` SMs at `mhz`: SMs x 8192
    flop per clock (one 128 x 256 x 16 MMA every 128 cycles per SM; the
    8192^3 capture in profiles/ reads 8060 flop per tensor-active cycle)."""
    return sms * SM_BF16_FLOP_PER_CLK * mhz * 1e6 / 1e12


def workload_record(name, sk, dev, pk, steps, warmup, flush):
    """One of the other configurations (FP32, FP8, grouped, autograd),
    measured like the sweep (inputs resident, L2 flushed before every timed
    run, CUDA events, median of `steps`), each next to its data-parallel
    counterpart.  Returns a record with per-case rows and the roofline of
    the dominant case."""
    auto, dp = sk.Config(), sk.Config(mode="dp")
    rows = []
    if name == "fp8":
        peak = 2 * pk["bf16"]
        peak_note = "2 x measured bf16 burst (no FP8 measurement available)"
        for i, (M, N, K) in enumerate(workloads.FP8_SHAPES):
            xa = workloads.device_normal((M, K), seed=2000 + 2 * i, device=dev)
            xb = workloads.device_normal((N, K), seed=2001 + 2 * i, device=dev)
            qa, sa = sk.quantize_e4m3(xa)
            qb, sb = sk.quantize_e4m3(xb)
            del xa, xb
            A, Bm = qa.view(torch.float8_e4m3fn), qb.view(torch.float8_e4m3fn).t()
            C = torch.empty(M, N, dtype=torch.bfloat16, device=dev)
            for cfg in (auto, dp):
                for _ in range(warmup):
                    sk.gemm(A, Bm, C, scale_a=sa, scale_b=sb, config=cfg)
            t = _timed_region(lambda: sk.gemm(A, Bm, C, scale_a=sa, scale_b=sb, config=auto), steps, flush)
            tdp = _timed_region(lambda: sk.gemm(A, Bm, C, scale_a=sa, scale_b=sb, config=dp), steps, flush)
            rows.append((f"{M}x{N}x{K} e4m3", workloads.gemm_flops(M, N, K), t, tdp))
        desc = "FP8 E4M3 per-tensor scaled, FP32 accumulate, BF16 out: " + " ".join(
            f"({m},{n},{k})" for m, n, k in workloads.FP8_SHAPES)
    elif name == "grouped":
        peak, peak_note = pk["bf16"], "measured bf16 burst"
        shapes = workloads.grouped_shapes(count=64, seed=0)
        As, Bs, Cs = [], [], []
        for i, (M, N, K) in enumerate(shapes):
            As.append(workloads.device_uniform((M, K), seed=3000 + 2 * i, device=dev))
            Bs.append(workloads.device_uniform((N, K), seed=3001 + 2 * i, device=dev).t())
            Cs.append(torch.empty(M, N, dtype=torch.bfloat16, device=dev))
        graphs = {}
        for gname, cfg in (("auto", auto), ("dp", dp)):
            sk.grouped_gemm(As, Bs, Cs, config=cfg)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    sk.grouped_gemm(As, Bs, Cs, config=cfg)
            torch.cuda.current_stream().wait_stream(s)
            graphs[gname] = g
        # per-problem launches (one graph of 64 launches), the library's default each
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for a, b, c in zip(As, Bs, Cs):
                sk.gemm(a, b, c)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                for a, b, c in zip(As, Bs, Cs):
                    sk.gemm(a, b, c)
        torch.cuda.current_stream().wait_stream(s)
        graphs["separate"] = g
        for gg in graphs.values():
            for _ in range(warmup):
                gg.replay()
        f = sum(workloads.gemm_flops(*x) for x in shapes)
        t = _timed_region(graphs["auto"].replay, steps, flush)
        tdp = _timed_region(graphs["dp"].replay, steps, flush)
        tsep = _timed_region(graphs["separate"].replay, steps, flush)
        rows.append(("grouped 64 (one launch)", f, t, tdp))
        rows.append(("64 separate launches", f, tsep, tsep))
        desc = ("grouped BF16: 64 problems, M log-uniform [64,4096], N,K from {1024,2048,4096,7168}, "
                "one persistent launch replayed from a CUDA graph")
    elif name == "autograd":
        peak, peak_note = pk["bf16"], "measured bf16 burst"
        M, N, K = workloads.AUTOGRAD_SHAPE
        A = workloads.device_uniform((M, K), seed=4000, device=dev).requires_grad_(True)
        Bm = workloads.device_uniform((N, K), seed=4001, device=dev).t().detach().requires_grad_(True)
        G = workloads.device_normal((M, N), seed=4002, device=dev, dtype=torch.bfloat16)

        def step(cfg):
            A.grad = None
            Bm.grad = None
            C = sk.sk_matmul(A, Bm, cfg)
            C.backward(G)

        for cfg in (auto, dp):
            for _ in range(warmup):
                step(cfg)
        f = 3 * workloads.gemm_flops(M, N, K)
        t = _timed_region(lambda: step(auto), steps, flush)
        tdp = _timed_region(lambda: step(dp), steps, flush)
        rows.append((f"{M}x{N}x{K} fwd+bwd", f, t, tdp))
        desc = "autograd BF16 layer: forward C=A*B plus backward dA=dC*B^T, dB=A^T*dC"
    elif name.startswith("f32"):
        # The library runs FP32 problems with K-major operands as 3xTF32 on
        # the tensor cores: three TF32 products per k-step at half the BF16
        # rate, so its useful peak is the measured BF16 peak / 2 / 3.  The
        # FFMA kernel's row is context (not in the totals), against the
        # derived FFMA peak: SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = pk["bf16"] / 2 / 3
        peak_note = (f"3xTF32: {pk['source']} bf16 burst {pk['bf16']} / 2 (TF32 rate) / 3 (products); "
                     f"FFMA row: {sms} SMs x 128 lanes x 2 flop x 2.07 GHz (derived)")
        ffma_peak = sms * 128 * 2 * 2.07e9 / 1e12
        M, N, K = (workloads.FP32_SMALL[x] for x in ("M", "N", "K"))
        if ":" in name:
            M, N, K = (int(x) for x in name.split(":", 1)[1].split(","))
        A = workloads.device_uniform((M, K), seed=5000, device=dev, dtype=torch.float32)
        Bm = workloads.device_uniform((N, K), seed=5001, device=dev, dtype=torch.float32).t()
        C = torch.empty(M, N, dtype=torch.float32, device=dev)
        ff, ffdp = sk.Config(f32_kernel="ffma"), sk.Config(mode="dp", f32_kernel="ffma")
        for cfg in (auto, dp, ff, ffdp):
            for _ in range(warmup):
                sk.gemm(A, Bm, C, config=cfg)
        t = _timed_region(lambda: sk.gemm(A, Bm, C, config=auto), steps, flush)
        tdp = _timed_region(lambda: sk.gemm(A, Bm, C, config=dp), steps, flush)
        rows.append((f"{M}x{N}x{K} f32 (3xTF32)", workloads.gemm_flops(M, N, K), t, tdp))
        t = _timed_region(lambda: sk.gemm(A, Bm, C, config=ff), steps, flush)
        tdp = _timed_region(lambda: sk.gemm(A, Bm, C, config=ffdp), steps, flush)
        rows.append((f"ffma kernel {M}x{N}x{K} f32", workloads.gemm_flops(M, N, K), t, tdp, ffma_peak))
        desc = (f"FP32 {M}x{N}x{K}, A row-major, B column-major, uniform[-1,1]; 128x128 tiles, "
                "3xTF32 tensor-core kernel (FFMA kernel as context)")
    else:
        raise ValueError(name)
    if ws_status(sk, dev) != 0:
        raise RuntimeError("device status")
    ctx = ("64 separate", "ffma kernel")   # context rows, not in the totals
    main = [r for r in rows if not r[0].startswith(ctx)]
    tot_f = sum(r[1] for r in main)
    tot_t = sum(r[2] for r in main)
    tot_dp = sum(r[3] for r in main)
    dom = max(main, key=lambda r: r[2])
    achieved = dom[1] / dom[2] / 1e9
    return {
        "workload": desc, "steps": steps, "warmup": warmup,
        "dtype": {"fp8": "e4m3"}.get(name, "f32" if name.startswith("f32") else "bf16"),
        "value": round(tot_f / (tot_t / 1e3) / 1e12, 2), "unit": UNIT, "ms": round(tot_t, 4),
        "dp_baseline": {"value": round(tot_f / (tot_dp / 1e3) / 1e12, 2), "unit": UNIT, "ms": round(tot_dp, 4)},
        "sk_over_dp": round(tot_dp / tot_t, 3),
        "rows": [{"case": r[0], "ms": round(r[2], 4), "us": round(1e3 * r[2], 2), "dp_us": round(1e3 * r[3], 2),
                  "tflops": round(r[1] / r[2] / 1e9, 2),
                  "pct_peak": round(100 * r[1] / r[2] / 1e9 / (r[4] if len(r) > 4 else peak), 1),
                  "dp_ms": round(r[3], 4),
                  "dp_tflops": round(r[1] / r[3] / 1e9, 1)} for r in rows],
        "roofline": {"bound": "tensor", "case": dom[0], "achieved": round(achieved, 1), "peak": round(peak, 1),
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "peak_source": peak_note},
        "peak": {"value": peak, "source": peak_note},
        "l2": "flushed (write then read 256 MB) before every timed run",
    }


def run_workload(args, world, rank, local):
    """One of the other configurations on its own (``--workload``)."""
    import paper_2407_00044_gb300 as sk
    dev = torch.device("cuda", torch.cuda.current_device())
    pk = peaks()
    flushbuf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush():
        flushbuf.fill_(1.0)
        torch.sum(flushbuf, dim=0, out=sink)

    steps = max(3, min(args.steps, 50))
    name = args.workload
    if name == "f32" and args.only:
        name = "f32:" + args.only
    rec = workload_record(name, sk, dev, pk, steps, args.warmup, flush)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": rec["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
        "config": {"workload": rec["workload"], "l2": rec["l2"]},
        "dp_baseline": rec["dp_baseline"], "rows": rec["rows"], "roofline": rec["roofline"], "peak": rec["peak"],
    }


def ws_status(sk, dev):
    return sk.default_workspace(dev).status()


# -------------------------------------------------------- CPU oracle arm
def cpu_baseline(seconds: float = 12.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the sweep:
    the first R rows of every sweep problem with full N and K, R chosen from
    a short calibration so the whole sample takes about ``seconds``."""
    import numpy as np

    import oracle
    threads = oracle.max_threads()
    rng_seed = 7

    def operands(R, N, K, seed):
        # A row-major, B column-major (K contiguous), as in the GPU workload
        a = workloads.uniform((R, K), seed=seed).to(torch.bfloat16)
        b = workloads.uniform((N, K), seed=seed + 1).to(torch.bfloat16)
        return oracle.to_f64(a), oracle.to_f64(b).T

    # calibration: one row per thread of the first problem
    M, N, K = workloads.BF16_SWEEP[0]
    a64, b64 = operands(threads, N, K, rng_seed)
    t0 = time.perf_counter()
    oracle.gemm(a64, b64, threads=threads)
    rate = workloads.gemm_flops(threads, N, K) / max(1e-6, time.perf_counter() - t0)
    budget = rate * seconds / len(workloads.BF16_SWEEP)
    done_flops = 0
    t_total = 0.0
    rows_used = []
    for i, (M, N, K) in enumerate(workloads.BF16_SWEEP):
        # whole multiples of the thread count, so every thread has rows
        R = int(budget // (2 * N * K)) // threads * threads
        R = int(max(threads, min(M, R)))
        a64, b64 = operands(R, N, K, rng_seed + 10 * i)
        t0 = time.perf_counter()
        oracle.gemm(a64, b64, threads=threads)
        t_total += time.perf_counter() - t0
        done_flops += workloads.gemm_flops(R, N, K)
        rows_used.append(R)
    rate_all = done_flops / t_total
    # one thread, on the first problem's first rows (about 2 s)
    M, N, K = workloads.BF16_SWEEP[0]
    R1 = max(1, int(rate_all / threads * 2.0 // (2 * N * K)))
    a64, b64 = operands(R1, N, K, rng_seed)
    t0 = time.perf_counter()
    oracle.gemm(a64, b64, threads=1)
    rate_one = workloads.gemm_flops(R1, N, K) / (time.perf_counter() - t0)
    # the FP32 problem (384 x 384 x 2048) in full
    f = workloads.FP32_SMALL
    a32 = oracle.to_f64(workloads.uniform((f["M"], f["K"]), seed=rng_seed))
    b32 = oracle.to_f64(workloads.uniform((f["N"], f["K"]), seed=rng_seed + 1)).T
    t0 = time.perf_counter()
    oracle.gemm(a32, b32, threads=threads)
    t_fp32 = time.perf_counter() - t0
    sweep_flops = sum(workloads.gemm_flops(*x) for x in workloads.BF16_SWEEP)
    return {"value": round(rate_all / 1e12, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first R rows (full N, K) of each sweep problem, R = " + ",".join(map(str, rows_used)) +
                      f"; FP64 triple loop with |A||B| scale; {round(t_total, 1)} s",
            "seconds": round(t_total, 2),
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "single_thread": {"value": round(rate_one / 1e12, 6), "unit": UNIT,
                              "sample": f"first {R1} rows of {M}x{N}x{K}"},
            "fp32_384x384x2048_full_s": round(t_fp32, 3),
            "sweep_full_s_extrapolated": round(sweep_flops / rate_all, 1)}


def cpu_model() -> str:
    """The host CPU's model name (x86 'model name', or the Arm part number)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model name", "Hardware"):
        for line in txt.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    parts = sorted({line.split(":", 1)[1].strip() for line in txt.splitlines() if line.startswith("CPU part")})
    impl = sorted({line.split(":", 1)[1].strip() for line in txt.splitlines() if line.startswith("CPU implementer")})
    if parts:
        return f"{platform.machine()} implementer {','.join(impl)} part {','.join(parts)}"
    return platform.machine()


def run_reference(args, world, rank):
    if rank != 0:
        return None
    # each step is a bounded oracle sample; the whole run stays within ~2.5 minutes
    per_step = max(0.2, min(args.ref_step_seconds, 150.0 / max(1, args.steps + args.warmup)))
    # warm-up steps (untimed), then timed steps, each a bounded oracle sample
    for _ in range(args.warmup):
        cpu_baseline(seconds=per_step)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(seconds=per_step)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(wall / max(1, args.steps) * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded uniform[-1,1] rounded to BF16 (numpy Philox)",
        "config": {"workload": WORKLOAD, "sample": last["sample"]},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=3.0)
    ap.add_argument("--only", default="", help="M,N,K: time this one problem instead of the sweep "
                    "(with --workload f32: instead of 384,384,2048)")
    ap.add_argument("--mode", default="auto", choices=["auto", "dp", "sk", "hybrid1", "hybrid2"])
    ap.add_argument("--fixup", default="owner", choices=["owner", "last_arriver", "split", "split_cluster"],
                    help="fixup of the Stream-K arm ('owner' lets the library choose among all)")
    ap.add_argument("--num-ctas", type=int, default=0, help="CTAs of the Stream-K arm (0 = library)")
    ap.add_argument("--tile", default="", help="tile of the Stream-K arm as MxN, e.g. 256x256 (default: library)")
    ap.add_argument("--no-dp", dest="dp", action="store_false", help="skip the data-parallel baseline")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false", help="skip the host-buffer run")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the FP32 / FP8 / grouped / autograd configurations in the default run")
    ap.add_argument("--no-search", dest="search", action="store_false",
                    help="skip timing every fixed tile/stages/mode candidate of the sweep shapes")
    ap.add_argument("--search-steps", type=int, default=20)
    ap.add_argument("--workload", default="sweep", choices=["sweep", "fp8", "grouped", "autograd", "f32"],
                    help="sweep (default, the headline) or one of the other configurations")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        if world > 1 or rank != 0:
            args.cpu_baseline = args.cpu_baseline and rank == 0 and world == 1
        line = run_ours(args, world, rank, local) if args.workload == "sweep" else run_workload(args, world, rank, local)
    if line is not None and rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
