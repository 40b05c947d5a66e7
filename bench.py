"""Benchmark of the row-skipping outer-product SpMM on one GB300.

Workload (conv-layer-shaped sweep, seed 1): A = 512 x 4608 (512 output x 512
input channels x 3 x 3) magnitude-pruned N(0,1) at sparsity
{50, 70, 90, 95, 99, 99.8}%, B = 4608 x 3136 post-ReLU activations
(half-normal, 50% zeros), C = 512 x 3136 FP32.  One step = the six SpMMs, one
per sparsity, each with its own B.  Two such input sets alternate between steps
(~430 MB with BF16 B, > the 129 MB L2), so no L2 flush is needed.

Headline form: A pre-packed in BF16 (Alg. 1 on the device), B in BF16, FP32
accumulation, schedule from the learned selector when its trained weights
ship with the package (else the analytic rule; the step under the analytic
rule is timed beside it).  Reported beside it: the plain FP32 form, cuSPARSE
CSR SpMM and cuBLAS dense GEMM (both through torch), 64 uneven layers batched
vs separate, the end-to-end call with host buffers, per-kernel shares (from
the library's own plan of each call), the roofline of the kernel with the
largest share and the oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPARSITIES = [0.5, 0.7, 0.9, 0.95, 0.99, 0.998]
M, K, N = 512, 4608, 3136
SEED = 1
METRIC = "SpMM 2·nnz·N GFLOP/s & HBM GB/s vs roofline; BF16/learned-tile vs plain FP32"
WORKLOAD = ("conv-layer SpMM sweep: A 512x4608 magnitude-pruned at "
            "{50,70,90,95,99,99.8}%, B 4608x3136 post-ReLU, C 512x3136 FP32, seed 1")
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="rosko", choices=["rosko", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the comparison legs (FP32, cuSPARSE, cuBLAS, batched, other "
                         "schedules)")
    ap.add_argument("--case", type=float, default=None,
                    help="profiling: run only the SpMM of this sparsity (BF16 and FP32 forms)")
    ap.add_argument("--autotune", action="store_true",
                    help="with --case: also run the autotuner and print every candidate's time")
    ap.add_argument("--schedule", default="analytic", choices=["analytic", "learned", "autotune"],
                    help="schedule of the timed step (the other two are timed beside it)")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)
    return a


# nominal HBM3e bandwidth of a GB300 (the measured copy peak is the roofline)
NOMINAL_HBM_GBS = 7900.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0,
                "source": "fallback"}


def make_inputs(stream_id: int):
    """A_s (FP32, pruned) and B_s (FP32 post-ReLU) for each sparsity."""
    from paper_2307_03930_gb300 import inputs as gen
    As, Bs = [], []
    for i, s in enumerate(SPARSITIES):
        ra = gen.rng_for(SEED, 1000 + i)
        As.append(gen.magnitude_prune(gen.normal((M, K), ra), s))
        rb = gen.rng_for(SEED, 2000 + 10 * stream_id + i)
        Bs.append(gen.relu_normal((K, N), rb))
    return As, Bs


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def traffic_for(kernel_key: str, src_files):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel_key)
    if not e:
        return None
    h = hashlib.sha256()
    for s in src_files:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    if e.get("src_sha256") != h.hexdigest():
        return None
    return e.get("dram_bytes_per_launch")


def src_sha(src_files):
    h = hashlib.sha256()
    for s in src_files:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# sources whose hash keys a committed DRAM-traffic figure (profiles/traffic.json)
KERNEL_SRC = {
    "dense_panel_kernel": ["paper_2307_03930_gb300/csrc/spmm_dense_tc.cu",
                           "paper_2307_03930_gb300/csrc/tc_common.cuh",
                           "paper_2307_03930_gb300/csrc/common.cuh"],
    "rowdirect_kernel": ["paper_2307_03930_gb300/csrc/spmm_sparse.cu",
                         "paper_2307_03930_gb300/csrc/common.cuh"],
}


# ----------------------------------------------------------------------------
# The oracle on the host cores: one worker process per core (started with
# `spawn`, since the parent has used the GPU), each holding the sweep's inputs
# and running the oracle as it stands on the row samples it is handed.
_W = {}


def _oracle_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    _W["inputs"] = make_inputs(0)


def _oracle_rows(task):
    """Oracle rows of one sparsity; returns their flops (2 nnz N)."""
    from oracle.spmm import spmm
    i, rows = task
    As, Bs = _W["inputs"]
    spmm(As[i], Bs[i], rows=np.asarray(rows))
    return 2.0 * float(np.count_nonzero(As[i][np.asarray(rows)])) * N


def _oracle_ready(_):
    return "inputs" in _W


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - not Linux
        return os.cpu_count() or 1


def oracle_pool():
    import multiprocessing as mp
    cores = host_cores()
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init)
    # every worker has built its inputs before anything is timed
    while not all(pool.map(_oracle_ready, range(4 * cores), chunksize=1)):
        pass
    return pool, cores


def cpu_baseline(budget_s: float = 12.0):
    """The oracle as it stands, on a bounded row sample of every sparsity,
    spread over all host cores (rows of a sparsity, 4 at a time, dealt to the
    workers; the sample ends once `budget_s` seconds of wall time have
    passed)."""
    pool, cores = oracle_pool()
    try:
        rng = np.random.default_rng(0)
        order = rng.permutation(M)
        tasks = [(i, order[j:j + 4].tolist()) for j in range(0, M, 4)
                 for i in range(len(SPARSITIES))]
        flops = 0.0
        rows_done = {s: 0 for s in SPARSITIES}
        t0 = time.perf_counter()
        t_end = t0
        for (i, rows), f in zip(tasks, pool.imap(_oracle_rows, tasks, chunksize=1)):
            flops += f
            rows_done[SPARSITIES[i]] += len(rows)
            t_end = time.perf_counter()
            if t_end - t0 > budget_s:
                break
        dt = t_end - t0
    finally:
        pool.terminate()
        pool.join()
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": ("rows " + ", ".join(f"{int(round(s * 1000)) / 10}%:{rows_done[s]}/{M}"
                                           for s in SPARSITIES)
                       + f" of the sweep, FP64 numpy oracle, {cores} worker processes, "
                         f"{dt:.1f} s")}


def run_reference(args, rank, world):
    """The reference arm: the oracle on all host cores, each step a bounded
    sample of the sweep (per sparsity, 2 rows per worker)."""
    if rank != 0:
        return
    steps = max(1, args.steps)
    warm = args.warmup
    pool, cores = oracle_pool()
    t_total = 0.0
    flops = 0.0
    try:
        for it in range(warm + steps):
            base = (it * 2 * cores) % M
            tasks = [(i, [(base + 2 * w) % M, (base + 2 * w + 1) % M])
                     for i in range(len(SPARSITIES)) for w in range(cores)]
            t0 = time.perf_counter()
            f = sum(pool.map(_oracle_rows, tasks, chunksize=1))
            dt = time.perf_counter() - t0
            if it >= warm:
                t_total += dt
                flops += f
    finally:
        pool.terminate()
        pool.join()
    v = flops / t_total / 1e9
    sample = f"{2 * cores} rows of each of the 6 sparsities per step ({cores} workers x 2 rows)"
    line = {"metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": world, "steps": steps,
            "warmup": warm, "ms_per_step": t_total / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample,
                       "parallelism": f"host, {cores} cores (one oracle process per core)"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2307_03930_gb300 import rosko

    if args.case is not None:
        profile_case(args, rosko, torch)
        return

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    rosko.lib()  # loud failure if the CUDA library is missing

    pk = peaks()
    # ---------------- inputs: two alternating sets, packed once ----------------
    sets = []
    for sid in range(2):
        As, Bs = make_inputs(sid) if sid == 0 else (sets[0]["A_np"], make_inputs(1)[1])
        entry = {"A_np": As, "B_np": Bs}
        entry["B16"] = [torch.from_numpy(b).to(dev).to(torch.bfloat16) for b in Bs]
        entry["C"] = [torch.empty((M, N), dtype=torch.float32, device=dev) for _ in SPARSITIES]
        sets.append(entry)
    handles16 = [rosko.rosko_pack(torch.from_numpy(a).to(dev), rosko.BF16) for a in sets[0]["A_np"]]
    infos = [h.info() for h in handles16]
    nnz = [i["nnz"] for i in infos]
    flops_step = sum(2.0 * z * N for z in nnz)
    stream = torch.cuda.current_stream()
    # schedule of the timed step: the library's default (analytic rule), or
    # the learned selector / the autotuner (their choice is made and cached
    # per handle on the first, untimed call); the other forms are timed beside
    learned_ok = False
    try:
        from paper_2307_03930_gb300 import selector as sel
        if os.path.exists(sel.WEIGHTS):
            sel.install()
            learned_ok = True
    except Exception as e:  # pragma: no cover - weights unreadable
        print(f"selector not installed: {e}", file=sys.stderr)
    tile, form = None, "analytic tile"
    if args.schedule == "learned" and learned_ok:
        tile, form = rosko.make_tile(mode=rosko.SCHED_LEARNED), "learned tile (MLP selector)"
    elif args.schedule == "autotune":
        tile, form = rosko.make_tile(mode=rosko.SCHED_AUTOTUNE), "autotuned tile"

    def step(t, hs=handles16, key="B16", tl=None):
        S = sets[t % 2]
        for i in range(len(SPARSITIES)):
            rosko.rosko_spmm(hs[i], S[key][i], S["C"][i], tile=tl if tl is not None else tile)

    for t in range(args.warmup):
        step(t)
    torch.cuda.synchronize()
    # The step (six SpMMs) is captured once per input set as a CUDA graph and
    # replayed: per-call host work (argument checks, tensor-map encoding) stays
    # out of the timed region, as in a deployed graph.
    graphs = []
    launches_per_step = None
    for sid in range(2):
        g = torch.cuda.CUDAGraph()
        l0 = rosko.rosko_kernel_launches()
        with torch.cuda.graph(g):
            step(sid)
        launches_per_step = rosko.rosko_kernel_launches() - l0
        graphs.append(g)
    for t in range(args.warmup):
        graphs[t % 2].replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        start.record(stream)
        for t in range(args.steps):
            graphs[t % 2].replay()
        end.record(stream)
        torch.cuda.synchronize()
    launches = launches_per_step * args.steps
    elapsed_ms = max_over_ranks(start.elapsed_time(end), dist if world > 1 else None, dev)
    # per-kernel device time: each SpMM alone, its B cycling through the six
    # distinct B buffers of one input set (~174 MB, > L2) so no call finds
    # its B in L2
    per_kernel_ms = [cycled_time(lambda j, i=i: rosko.rosko_spmm(
        handles16[i], sets[0]["B16"][j], sets[0]["C"][j], tile=tile), torch)
        for i in range(len(SPARSITIES))]
    ms_step = elapsed_ms / args.steps
    value = job_value(flops_step, args.steps, world, elapsed_ms)
    status = rosko.rosko_device_status(clear=True)
    # which kernel each SpMM runs (the library's own plan of the call)
    plans = [rosko.rosko_spmm_plan(handles16[i], sets[0]["B16"][i], sets[0]["C"][i], tile=tile)
             for i in range(len(SPARSITIES))]
    # the step under each schedule (graph replays of one input set): the
    # analytic rule, the learned selector, the per-shape autotuner (its search
    # runs on the first, uncaptured call of each handle and is cached)
    forms_ms = {"analytic": graph_time(lambda: step(0, tl=rosko.make_tile()), torch, reps=20)}
    if learned_ok and not args.no_extras:
        forms_ms["learned"] = graph_time(lambda: step(0, tl=rosko.make_tile(mode=rosko.SCHED_LEARNED)),
                                         torch, reps=20)
        forms_ms["learned_choices"] = [rosko.rosko_spmm_plan(
            handles16[i], sets[0]["B16"][i], sets[0]["C"][i],
            tile=rosko.make_tile(mode=rosko.SCHED_LEARNED))["tile"] for i in range(len(SPARSITIES))]
    if not args.no_extras:
        forms_ms["autotune"] = graph_time(
            lambda: step(0, tl=rosko.make_tile(mode=rosko.SCHED_AUTOTUNE)), torch, reps=20)
        # the six independent layers as one rosko_spmm_batched call (one
        # tensor-core launch for the five dense layers, one row-direct launch)
        forms_ms["batched_call"] = graph_time(
            lambda: rosko.rosko_spmm_batched(handles16, sets[0]["B16"], sets[0]["C"]), torch,
            reps=20)

    # ---------------- per-sparsity figures and the roofline -------------------
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak_tflops = sms * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    per = []
    for i, s in enumerate(SPARSITIES):
        inf = infos[i]
        bytes_alg = inf["bytes"] + inf["touched_k"] * N * 2 + M * N * 4
        t = per_kernel_ms[i] * 1e-3
        pl = plans[i]
        kern = ("dense_panel_kernel" if pl["sparse_panels"] == 0 else
                "rowdirect_kernel" if pl["dense_tiles"] == 0 else "dense_panel+rowdirect")
        if pl["dense_tiles"] == 0 and pl["order"] != 4:
            kern = f"sparse_spmm_kernel(order {pl['order']})"
        gflops = 2.0 * nnz[i] * N / t / 1e9
        # arithmetic peak of the kernel: the BF16 tensor peak for the
        # tensor-core path, the FP32 FFMA peak for the CUDA-core traversals
        arith = pk["bf16_tflops"] if kern.startswith("dense") else fp32_peak_tflops
        row = {"sparsity": s, "nnz": nnz[i], "ms": per_kernel_ms[i], "kernel": kern,
               "plan": pl, "gflops": gflops, "alg_bytes": bytes_alg,
               "hbm_gbs": bytes_alg / t / 1e9,
               "hbm_frac": bytes_alg / t / 1e9 / pk["hbm_gbs"],
               "hbm_frac_nominal": bytes_alg / t / 1e9 / NOMINAL_HBM_GBS,
               "alu_frac": gflops / 1e3 / arith, "alu_peak_tflops": arith}
        if pl["dense_tiles"] > 0:
            # the work the tensor cores do: every row of the dense tiles
            # times K times N, zeros included
            dense_rows = min(M, pl["dense_tiles"] * 128)
            row["tensor_work_tflops"] = 2.0 * dense_rows * K * N / t / 1e12
            row["tensor_work_frac"] = row["tensor_work_tflops"] / pk["bf16_tflops"]
        per.append(row)
    # the dominant kernel: largest share of the per-kernel time of a step
    kinds = {}
    for r in per:
        k = kinds.setdefault(r["kernel"], {"launches_per_step": 0, "ms": 0.0, "alg_bytes": 0.0,
                                           "alg_flops": 0.0})
        k["launches_per_step"] += 1
        k["ms"] += r["ms"]
        k["alg_bytes"] += r["alg_bytes"]
        k["alg_flops"] += 2.0 * r["nnz"] * N
    tot_ms = sum(k["ms"] for k in kinds.values())
    for k in kinds.values():
        k["share"] = k["ms"] / tot_ms
    dom_name = max(kinds, key=lambda k: kinds[k]["ms"])
    dk = kinds[dom_name]
    # bound: whichever of algorithmic bytes at HBM peak and algorithmic flops
    # at the kernel's arithmetic peak takes longer
    arith_peak = pk["bf16_tflops"] if dom_name.startswith("dense") else fp32_peak_tflops
    t_arith = dk["alg_flops"] / (arith_peak * 1e12)
    t_hbm = dk["alg_bytes"] / (pk["hbm_gbs"] * 1e9)
    sec = dk["ms"] * 1e-3
    if t_arith > t_hbm:
        roof = {"bound": "tensor" if dom_name.startswith("dense") else "alu",
                "achieved": dk["alg_flops"] / sec / 1e12, "peak": arith_peak, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": dk["alg_bytes"] / sec / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_for(dom_name, KERNEL_SRC.get(dom_name, []))
    roof["kernel"] = dom_name
    roof["launches_per_step"] = dk["launches_per_step"]
    roof["per_launch_ms"] = dk["ms"] / dk["launches_per_step"]
    roof["alg_bytes_per_launch"] = dk["alg_bytes"] / dk["launches_per_step"]
    if dom_name.startswith("dense"):
        # beside the roofline of the algorithmic work: the tensor cores'
        # own work (dense tiles, zeros included) against the BF16 peak
        tw = [r["tensor_work_tflops"] * r["ms"] for r in per
              if r["kernel"] == dom_name and "tensor_work_tflops" in r]
        roof["tensor_work_frac"] = sum(tw) / dk["ms"] / pk["bf16_tflops"]
    roof["peak_source"] = (f"{pk['source']} (MEASURED_PEAKS.json)" if roof["bound"] in ("hbm", "tensor")
                           else f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x "
                                f"{pk['sm_max_mhz']:.0f} MHz")

    extras = {}
    if not args.no_extras:
        extras = comparison_legs(rosko, torch, dev, sets, infos, stream)
        extras["batched_uneven_layers"] = batched_leg(rosko, torch, dev)
        extras["training_step"] = training_leg(rosko, torch, dev, sets)
        extras["pack"] = pack_leg(rosko, torch, dev, sets)
        extras["other_configs"] = other_configs_leg(rosko, torch, dev)

    # ---------------- end to end: host buffers through the C-ABI -----------------
    e2e = end_to_end(rosko, torch, dev, sets, handles16, stream, flops_step, world, tile=tile)

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": f"BF16 A and B, FP32 accumulate, {form}",
                       "l2": f"inputs alternate between 2 sets of {2 * 6 * K * N * 2 / 1e6:.0f} MB "
                             "of BF16 B (> 129 MB L2), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "device_status": status,
            "kernels": kinds, "per_sparsity": per,
            "schedule": {"form": form, "step_ms_graph_by_schedule": forms_ms},
            "comparisons": extras}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def profile_case(args, rosko, torch):
    """One sparsity of the sweep, BF16 (schedule as in the bench) then FP32,
    `--steps` launches each after `--warmup`; prints the event time per launch."""
    from paper_2307_03930_gb300 import inputs as gen
    dev = torch.device("cuda", 0)
    i = min(range(len(SPARSITIES)), key=lambda j: abs(SPARSITIES[j] - args.case))
    A = gen.magnitude_prune(gen.normal((M, K), gen.rng_for(SEED, 1000 + i)), SPARSITIES[i])
    # six distinct B (> L2 together) so that timed calls read B from HBM
    Bs = [gen.relu_normal((K, N), gen.rng_for(SEED, 2000 + 10 * j + i)) for j in range(6)]
    Ad = torch.from_numpy(A).to(dev)
    out = {"sparsity": SPARSITIES[i]}
    forms = (("bf16", rosko.BF16, torch.bfloat16, None),
             ("bf16_colorder", rosko.BF16, torch.bfloat16, rosko.make_tile(order=1)),
             ("bf16_sparse_only", rosko.BF16, torch.bfloat16, rosko.make_tile(dense_split_pm=1001)),
             ("f32", rosko.F32, torch.float32, None),
             ("f32_colorder", rosko.F32, torch.float32, rosko.make_tile(order=1)))
    for name, code, bd, tile in forms:
        h = rosko.rosko_pack(Ad, code)
        Bd = [torch.from_numpy(B).to(dev).to(bd) for B in Bs]
        Cd = [torch.empty((M, N), device=dev) for _ in Bs]
        for _ in range(args.warmup):
            rosko.rosko_spmm(h, Bd[0], Cd[0], tile=tile)
        out[name + "_ms"] = cycled_time(lambda j: rosko.rosko_spmm(h, Bd[j], Cd[j], tile=tile),
                                        torch, reps=max(6, args.steps))
        if args.autotune and name in ("bf16", "f32"):
            best, times = rosko.rosko_autotune(h, Bd[0], Cd[0])
            out[name + "_autotuned_ms"] = min(t for t in times if t is not None)
            out[name + "_autotuned_tile"] = best.as_dict()
            out[name + "_candidates_ms"] = [None if t is None else round(t, 5) for t in times]
    print(json.dumps(out), flush=True)


def max_over_ranks(value: float, dist, device=None) -> float:
    """Barrier, then the maximum of `value` over all ranks (the slowest rank's
    time defines the job's time); identity without a process group."""
    import torch
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(flops_per_step_per_rank: float, steps: int, world: int, elapsed_ms: float) -> float:
    """Whole-job throughput in GFLOP/s: every rank runs the same per-rank work
    (weak scaling), timed by the slowest rank."""
    return world * flops_per_step_per_rank * steps / (elapsed_ms * 1e-3) / 1e9


def graph_time(fn, torch, reps=20):
    """Mean device time (ms) of `fn` (one library call) over `reps` calls
    captured in one CUDA graph; the inputs alternate between two sets inside
    the callers where it matters for L2."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    g.replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def cycled_time(fn, torch, reps=24, n_buf=6):
    """Mean device time (ms) of fn(j) over `reps` calls captured in one CUDA
    graph, j cycling over n_buf input buffers (chosen so their sum exceeds
    L2)."""
    for j in range(n_buf):
        fn(j)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for r in range(reps):
            fn(r % n_buf)
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    g.replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time(fn, torch, stream, reps=20, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def other_configs_leg(rosko, torch, dev):
    """The other fixed configurations, analytic schedule, CUDA-event graph
    timing with cycled B (> L2): plain FP32 1024 x 1024 x 1024 at 90%
    (uniform, seed 0), and the transformer-FFN shapes 11008 x 4096 and
    4096 x 11008 (K x 2048 tokens, magnitude-pruned at 70/90/95%, seed 2) in
    BF16 -> FP32 and INT8 -> INT32."""
    from paper_2307_03930_gb300 import inputs as gen
    out = {}
    rng = gen.rng_for(0)
    A = gen.sparse_weight(1024, 1024, 0.9, rng, "uniform")
    h = rosko.rosko_pack(torch.from_numpy(A).to(dev), rosko.F32)
    Bs = [torch.randn((1024, 1024), device=dev) for _ in range(40)]   # 160 MB
    Cs = [torch.empty((1024, 1024), device=dev) for _ in range(40)]
    ms = cycled_time(lambda j: rosko.rosko_spmm(h, Bs[j], Cs[j]), torch, reps=40, n_buf=40)
    out["c1_fp32_1024_s90"] = {"us": ms * 1e3, "gflops": 2.0 * h.info()["nnz"] * 1024 / ms / 1e6}
    del Bs, Cs, h
    for (Mx, Kx) in ((11008, 4096), (4096, 11008)):
        for s in (0.7, 0.9, 0.95):
            rng = gen.rng_for(2, Mx, int(round(s * 100)))
            A = gen.magnitude_prune(gen.normal((Mx, Kx), rng), s)
            Ad = torch.from_numpy(A).to(dev)
            nb = 3
            B16 = [torch.randn((Kx, 2048), device=dev).to(torch.bfloat16) for _ in range(nb)]
            B8 = [torch.randint(-127, 128, (Kx, 2048), device=dev, dtype=torch.int8)
                  for _ in range(nb)]
            C32 = [torch.empty((Mx, 2048), device=dev) for _ in range(nb)]
            C32i = [torch.empty((Mx, 2048), device=dev, dtype=torch.int32) for _ in range(nb)]
            h16 = rosko.rosko_pack(Ad, rosko.BF16)
            h8 = rosko.rosko_pack(Ad, rosko.I8)
            nnz = h16.info()["nnz"]
            key = f"c3_{Mx}x{Kx}x2048_s{int(round(s * 100))}"
            t16 = cycled_time(lambda j: rosko.rosko_spmm(h16, B16[j], C32[j]), torch, reps=6,
                              n_buf=nb)
            t8 = cycled_time(lambda j: rosko.rosko_spmm(h8, B8[j], C32i[j]), torch, reps=6,
                             n_buf=nb)
            out[key] = {"bf16_us": t16 * 1e3, "bf16_gflops": 2.0 * nnz * 2048 / t16 / 1e6,
                        "int8_us": t8 * 1e3, "int8_gops": 2.0 * h8.info()["nnz"] * 2048 / t8 / 1e6}
            del Ad, B16, B8, C32, C32i, h16, h8
    return out


def pack_leg(rosko, torch, dev, sets):
    """Device pack (Alg. 1, BF16 with dense copies) of each A of the sweep
    against cuSPARSE's dense -> CSR conversion (torch.to_sparse_csr) of the
    same FP32 matrix (the inspector cost of dynamic sparsity, Sec. 4.1);
    wall time per conversion, synchronised (the pack reads its sizes back)."""
    out = []
    for i, s in enumerate(SPARSITIES):
        A32 = torch.from_numpy(sets[0]["A_np"][i]).to(dev)
        ts = {}
        for name, fn in (("rosko_pack_bf16", lambda: rosko.rosko_pack(A32, rosko.BF16)),
                         ("rosko_pack_f32", lambda: rosko.rosko_pack(A32, rosko.F32)),
                         ("cusparse_dense_to_csr", lambda: A32.to_sparse_csr())):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                r = fn()
                torch.cuda.synchronize()
                del r
            ts[name + "_ms"] = (time.perf_counter() - t0) / 5 * 1e3
        out.append({"sparsity": s, **ts})
    return out


def comparison_legs(rosko, torch, dev, sets, infos, stream):
    """Plain FP32 form, cuSPARSE CSR and cuBLAS dense on the same shapes.  Each
    timed call cycles through the six distinct B buffers of one input set
    (> L2), like the timed step."""
    out = {"fp32_plain": [], "cusparse_csr_f32": [], "cublas_dense_bf16": []}
    B32 = [torch.from_numpy(b).to(dev) for b in sets[0]["B_np"]]
    B16 = sets[0]["B16"]
    Cs = sets[0]["C"]
    pk = peaks()
    out["footprint"] = []
    for i, s in enumerate(SPARSITIES):
        A32 = torch.from_numpy(sets[0]["A_np"][i]).to(dev)
        fl = 2.0 * infos[i]["nnz"] * N
        h32 = rosko.rosko_pack(A32, rosko.F32)
        i32 = h32.info()
        ms = cycled_time(lambda j: rosko.rosko_spmm(h32, B32[j], Cs[j]), torch)
        # the FP32 form's own roofline: FP32 packed A + touched FP32 B rows +
        # C, against the measured HBM peak
        b32 = i32["bytes"] + i32["touched_k"] * N * 4 + M * N * 4
        out["fp32_plain"].append({"sparsity": s, "ms": ms, "gflops": fl / ms / 1e6,
                                  "alg_bytes": b32, "hbm_gbs": b32 / ms / 1e6,
                                  "hbm_frac": b32 / ms / 1e6 / pk["hbm_gbs"]})
        # device footprint of the packed handles against dense and CSR storage
        nz = infos[i]["nnz"]
        out["footprint"].append({
            "sparsity": s, "bf16_handle_device_bytes": infos[i]["device_bytes"],
            "bf16_column_format_bytes": infos[i]["bytes"],
            "fp32_handle_device_bytes": i32["device_bytes"],
            "fp32_column_format_bytes": i32["bytes"],
            "dense_bf16_bytes": M * K * 2, "dense_fp32_bytes": M * K * 4,
            "csr_fp32_bytes": nz * 8 + (M + 1) * 4, "csr_bf16_bytes": nz * 6 + (M + 1) * 4})
        Acsr = A32.to_sparse_csr()
        cnt = [0]

        def csr():
            cnt[0] += 1
            torch.mm(Acsr, B32[cnt[0] % len(B32)])
        try:
            ms = _time(csr, torch, stream, reps=12)
            out["cusparse_csr_f32"].append({"sparsity": s, "ms": ms, "gflops": fl / ms / 1e6})
        except Exception as e:  # pragma: no cover
            out["cusparse_csr_f32"].append({"sparsity": s, "error": str(e)[:80]})
        A16 = A32.to(torch.bfloat16)
        ms = cycled_time(lambda j: torch.mm(A16, B16[j]), torch)
        out["cublas_dense_bf16"].append({"sparsity": s, "ms": ms, "gflops_alg": fl / ms / 1e6})
        del h32, Acsr
    del B32
    for k in list(out):
        if not isinstance(out[k], list):
            continue
        rows = [r for r in out[k] if "ms" in r]
        if rows:
            tot = sum(r["ms"] for r in rows)
            fl = sum(2.0 * infos[i]["nnz"] * N for i in range(len(rows)))
            out[k + "_sweep_gflops"] = fl / tot / 1e6
    r32 = out["fp32_plain"]
    tot = sum(r["ms"] for r in r32)
    byt = sum(r["alg_bytes"] for r in r32)
    out["fp32_roofline"] = {"bound": "hbm", "kernel": "rowdirect_kernel (FP32)",
                            "achieved": byt / tot / 1e6, "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": byt / tot / 1e6 / pk["hbm_gbs"],
                            "note": "whole FP32 sweep: algorithmic bytes / summed kernel time"}
    return out


def batched_leg(rosko, torch, dev, seed=3, count=64):
    """Uneven layers (64 SpMMs: M, K log-uniform in [64, 4096], N in
    [196, 12544], sparsity uniform in [0.70, 0.99], BF16): one
    rosko_spmm_batched call captured in a CUDA graph, with the analytic rule's
    tiles and with per-shape tiles from rosko_autotune, against 64 separate
    rosko_spmm calls captured in a graph and issued from the host; beside
    them the per-problem roofline sum, sum_i max(bytes_i / HBM peak,
    2 nnz_i N_i / BF16 peak)."""
    from paper_2307_03930_gb300 import inputs as gen
    pk = peaks()
    shapes = gen.c4_shapes(seed, count)
    hs, Bs, Cs, flops, roof_s = [], [], [], 0.0, 0.0
    for j, (M_, K_, N_, s_) in enumerate(shapes):
        A = gen.sparse_weight(M_, K_, s_, gen.rng_for(seed, 1, j), "uniform")
        h = rosko.rosko_pack(torch.from_numpy(A).to(dev), rosko.BF16)
        ldb = -(-N_ // 8) * 8
        Bb = torch.from_numpy(gen.relu_normal((K_, N_), gen.rng_for(seed, 2, j))).to(dev)
        Bbuf = torch.zeros((K_, ldb), dtype=torch.bfloat16, device=dev)
        Bbuf[:, :N_] = Bb.to(torch.bfloat16)
        hs.append(h)
        Bs.append(Bbuf[:, :N_])
        Cs.append(torch.empty((M_, N_), device=dev))
        inf = h.info()
        fl = 2.0 * inf["nnz"] * N_
        flops += fl
        byt = inf["bytes"] + inf["touched_k"] * N_ * 2 + M_ * N_ * 4
        roof_s += max(byt / (pk["hbm_gbs"] * 1e9), fl / (pk["bf16_tflops"] * 1e12))
    work_mb = sum(b.numel() * 2 + c.numel() * 4 for b, c in zip(Bs, Cs)) / 1e6
    tuned = [rosko.rosko_autotune(h, b, c)[0] for h, b, c in zip(hs, Bs, Cs)]

    def batched():
        rosko.rosko_spmm_batched(hs, Bs, Cs)

    def batched_tuned():
        rosko.rosko_spmm_batched(hs, Bs, Cs, tiles=tuned)

    def separate():
        for h, b, c in zip(hs, Bs, Cs):
            rosko.rosko_spmm(h, b, c)

    out = {"problems": count, "gflop": flops / 1e9, "working_set_mb": work_mb,
           "roofline_sum_ms": roof_s * 1e3}
    for name, fn in (("batched_graph", batched), ("batched_autotuned_graph", batched_tuned),
                     ("separate_graph", separate)):
        out[name + "_ms"] = graph_time(fn, torch, reps=5)
        out[name + "_gflops"] = flops / (out[name + "_ms"] * 1e-3) / 1e9
        out[name + "_roofline_frac"] = roof_s * 1e3 / out[name + "_ms"]
    for _ in range(2):
        separate()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        separate()
    b.record()
    torch.cuda.synchronize()
    out["separate_launches_ms"] = a.elapsed_time(b) / 5
    out["separate_launches_gflops"] = flops / (out["separate_launches_ms"] * 1e-3) / 1e9
    l0 = rosko.rosko_kernel_launches()
    batched()
    out["batched_kernel_launches"] = rosko.rosko_kernel_launches() - l0
    torch.cuda.synchronize()
    return out


def training_leg(rosko, torch, dev, sets):
    """The SpMMs of a pruned layer's training step (Sec. 5.4): the forward
    O = W X with the packed W, the input gradient dX = W^T dO with W^T packed
    by rosko_pack_transposed, and that re-pack itself (paid once per pruning
    epoch, when the mask changes), on the 512 x 4608 layer with 3136 columns,
    BF16, at 90% and 99%."""
    out = []
    dO = [torch.randn((M, N), device=dev).to(torch.bfloat16) for _ in range(6)]
    dX = [torch.empty((K, N), device=dev) for _ in range(6)]
    for i, s in enumerate(SPARSITIES):
        if s not in (0.9, 0.99):
            continue
        W = torch.from_numpy(sets[0]["A_np"][i]).to(dev)
        hT = rosko.rosko_pack_transposed(W, rosko.BF16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            h2 = rosko.rosko_pack_transposed(W, rosko.BF16)
            torch.cuda.synchronize()
            del h2
        repack_ms = (time.perf_counter() - t0) / 5 * 1e3
        nnz = hT.info()["nnz"]
        ms_t = cycled_time(lambda j: rosko.rosko_spmm(hT, dO[j], dX[j]), torch)
        plan = rosko.rosko_spmm_plan(hT, dO[0], dX[0])
        out.append({"sparsity": s, "transposed_spmm_ms": ms_t,
                    "transposed_spmm_gflops": 2.0 * nnz * N / ms_t / 1e6,
                    "transposed_dense_tiles": plan["dense_tiles"],
                    "transposed_sparse_panels": plan["sparse_panels"],
                    "repack_transposed_ms": repack_ms})
        del hT, W
    return out


def end_to_end(rosko, torch, dev, sets, handles, stream, flops_step, world, steps=50, tile=None):
    """Same metric through the C-ABI with pinned host buffers: per step the six
    B inputs are copied host->device, the SpMMs run, and the six C results are
    copied back (the packed weights stay resident, as for pre-packed inference
    weights, Sec. 4.1).  Three streams pipeline the layers: layer i+1's input
    copy and layer i-1's result copy overlap layer i's SpMM (events order
    each buffer's copy-in, SpMM and copy-out, also across steps)."""
    hB = [[torch.from_numpy(b).to(torch.bfloat16).pin_memory() for b in S["B_np"]] for S in sets]
    hC = [torch.empty((M, N), dtype=torch.float32).pin_memory() for _ in SPARSITIES]
    dB = [torch.empty((K, N), dtype=torch.bfloat16, device=dev) for _ in SPARSITIES]
    dC = [torch.empty((M, N), dtype=torch.float32, device=dev) for _ in SPARSITIES]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    n = len(SPARSITIES)
    ev_in = [torch.cuda.Event() for _ in range(n)]     # B_i on the device
    ev_mm = [torch.cuda.Event() for _ in range(n)]     # SpMM_i done (B_i free, C_i ready)
    ev_out = [torch.cuda.Event() for _ in range(n)]    # C_i copied back (C_i free)
    for i in range(n):
        for e in (ev_mm[i], ev_out[i]):
            e.record(stream)

    def one(t):
        for i in range(n):
            s_in.wait_event(ev_mm[i])              # previous step's SpMM_i read B_i
            with torch.cuda.stream(s_in):
                dB[i].copy_(hB[t % 2][i], non_blocking=True)
                ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            stream.wait_event(ev_out[i])           # previous step's C_i copied out
            rosko.rosko_spmm(handles[i], dB[i], dC[i], tile=tile, stream=stream)
            ev_mm[i].record(stream)
            s_out.wait_event(ev_mm[i])
            with torch.cuda.stream(s_out):
                hC[i].copy_(dC[i], non_blocking=True)
                ev_out[i].record(s_out)

    for t in range(3):
        one(t)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s_in.wait_event(a)
    for t in range(steps):
        one(t)
    stream.wait_stream(s_out)
    stream.wait_stream(s_in)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"value": world * flops_step / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
            "h2d_bytes_per_step": n * K * N * 2,
            "d2h_bytes_per_step": n * M * N * 4, "ms_per_step": ms,
            "steps": steps, "pipelining": "3 streams (copy-in, SpMM, copy-out)"}


if __name__ == "__main__":
    main()
