"""Benchmark of the memory-bound hot path on GB300.

One step = one pass over the full-HBM memory-bound workload:
  * int32 sum reduce of 2^30 values in [-1000, 1000] through the hierarchical
    view group(1024)[[block]].group(32)[[warp]][[thread]] (one scalar out),
  * FP32 inclusive scan of 2^28 values uniform in [-1, 1),
  * FP32 out-of-place transpose of a 16384 x 16384 N(0,1) matrix,
each through libdesc's C ABI, inputs resident in HBM.  value = algorithmic
bytes of the step (reduce 4 B/elem, scan 8 B/elem, transpose 8 B/elem) per
second.  Every input is larger than L2, so no flush is needed between steps.

--impl reference times the CPU oracle instead, on bounded samples of the same
workload, and prints the same line with "impl": "reference".
Under torchrun every rank runs its own replica (the ops are single-GPU; no
data-path collective); value sums the ranks' bytes over the slowest rank.
"""
from __future__ import annotations

import argparse
import datetime as dt
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HBM GB/s & % roofline (reduce/scan/transpose); matmul TFLOP/s at stated error"
WORKLOAD = "full-HBM memory-bound set: int32 reduce 2^30, FP32 inclusive scan 2^28, FP32 transpose 16384x16384"


def sizes(small):
    if small:   # for profiler captures: still larger than L2, a few hundred MB on the device
        return {"reduce_n": 1 << 26, "scan_n": 1 << 26, "T": 4096}
    return {"reduce_n": 1 << 30, "scan_n": 1 << 28, "T": 16384}


def op_bytes(sz):
    return {"reduce": 4 * sz["reduce_n"], "scan": 8 * sz["scan_n"], "transpose": 8 * sz["T"] * sz["T"]}


# Nominal GB300 figures (the data sheet's, not measured here): HBM3e 7.9 TB/s,
# dense BF16 tensor 2.25 PFLOP/s at the 2070 MHz maximum SM clock.
NOMINAL_HBM_GBS = 7900.0
NOMINAL_BF16_TFLOPS = 2250.0
NOMINAL_SM_MHZ = 2070.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def max_over_ranks(torch, ms, dev):
    """The slowest rank's time: every rank gets the maximum of the ranks' ms
    (the process group's backend decides the device of the reduction)."""
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def job_rate(world, step_bytes, steps, ms):
    """Whole-job GB/s: the bytes every rank moved in `steps` steps over the
    slowest rank's time (replicas: each rank runs the full step)."""
    return world * step_bytes * steps / (ms * 1e-3) / 1e9


def traffic_for(op):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source has changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == op:
            src = os.path.join(ROOT, "paper_2305_03448_gb300", "csrc", f[3])
            if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest()[:12] == f[2]:
                return float(f[1])
    return None


class Clocks:
    """nvidia-smi samples of this GPU while the timed region runs."""
    Q = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = (uuid or "").lower()
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self, t0, t1):
        if self.p is None:
            return None
        time.sleep(0.1)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[1].lower():
                continue
            try:
                ts = dt.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        win = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05] or rows
        sm = sorted(r[1] for r in win)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in win for i in range(4) if r[3][i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[2] for r in win), "reasons": reasons,
                "samples": len(win), "window": "timed" if len(win) < len(rows) or t1 - t0 > 0.05 else "run"}


def _gpu_uuid(torch, dev):
    u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    return str(u) if u else None


# --------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2305_03448_gb300 as D
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if args.generic:
        D.desc_force_generic(True)
    sz = sizes(args.small)
    nb = op_bytes(sz)
    Rn, Sn, T = sz["reduce_n"], sz["scan_n"], sz["T"]
    V = D
    red_ops = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
               ("select", V.THREAD, V.X)]
    red_grid, red_block = (Rn // 1024, 1, 1), (1024, 1, 1)

    xr = synth.ints_pm1000(Rn, seed=1 + rank, device=dev)
    xs = synth.uniform_grid(Sn, seed=2 + rank, device=dev)
    xt = synth.normal_f32(T * T, seed=3 + rank, device=dev).reshape(T, T)
    out_r = torch.empty(1, dtype=torch.int32, device=dev)
    out_s = torch.empty_like(xs)
    out_t = torch.empty(T, T, dtype=torch.float32, device=dev)

    def ws_for(kind):
        import ctypes
        n = ctypes.c_size_t(0)
        L = D.lib()
        if kind == "reduce":
            L.desc_reduce_workspace_size(ctypes.byref(D.make_view([Rn], red_ops)),
                                         ctypes.byref(D.make_exec(red_grid, red_block)), V.GRID, V.I32, ctypes.byref(n))
        else:
            L.desc_scan_workspace_size(ctypes.byref(D.make_view([Sn], [])), None, V.GRID, V.F32, ctypes.byref(n))
        return torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)

    ws_r, ws_s = ws_for("reduce"), ws_for("scan")
    stream = torch.cuda.current_stream(dev)

    def op_reduce(x=xr, out=out_r):
        D.desc_reduce(x, [Rn], red_ops, V.GRID, red_grid, red_block, out=out, ws=ws_r, stream=stream)

    def op_scan(x=xs, out=out_s, stream=stream):
        D.desc_scan(x, [Sn], [], V.GRID, out=out, ws=ws_s, stream=stream)

    def op_transpose(x=xt, out=out_t):
        D.desc_transpose(x, [T, T], [("transpose", 0)], out, [T, T], [], stream=stream)

    ops = [("reduce", op_reduce), ("scan", op_scan), ("transpose", op_transpose)]
    only = set(args.ops.split(",")) if args.ops else None
    if only:
        ops = [o for o in ops if o[0] in only]
    schedules = None
    if args.load_tune:
        D.desc_tune_load(args.load_tune)
        schedules = {"loaded": args.load_tune}
    elif not args.no_tune:
        red_view = dict(view=([Rn], red_ops), grid=red_grid, block=red_block, level=V.GRID)
        schedules = autotune_step(D, stream, {"reduce": (D.OP_REDUCE, D.I32, Rn, 0, xr, out_r, ws_r, red_view),
                                              "scan": (D.OP_SCAN, D.F32, Sn, 0, xs, out_s, ws_s, None),
                                              "transpose": (D.OP_TRANSPOSE, D.F32, T * T, T, xt, out_t, ws_s, None)},
                                  [name for name, _ in ops])
        if args.save_tune:
            D.desc_tune_save(args.save_tune)
    for _ in range(args.warmup):
        for _, f in ops:
            f()
    torch.cuda.synchronize(dev)
    status = D.desc_stream_status(stream)
    if status != 0:
        raise RuntimeError(f"device status {status} after warm-up")

    K = args.steps
    ev = {name: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
          for name, _ in ops}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(_gpu_uuid(torch, dev)) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.time()
    e0.record(stream)
    for k in range(K):
        for name, f in ops:
            a, b = ev[name][k]
            a.record(stream)
            f()
            b.record(stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop(t0, t1) if clocks else None
    ms = e0.elapsed_time(e1)
    if world > 1:
        ms = max_over_ranks(torch, ms, dev)
    status = D.desc_stream_status(stream)
    if status != 0:
        raise RuntimeError(f"device status {status} in the timed region")
    step_bytes = sum(nb[name] for name, _ in ops)
    value = job_rate(world, step_bytes, K, ms)
    per_op = {}
    for name, _ in ops:
        d = [a.elapsed_time(b) for a, b in ev[name]]
        avg = sum(d) / len(d)
        per_op[name] = {"ms": round(avg, 4), "GB/s": round(nb[name] / (avg * 1e-3) / 1e9, 1)}
    pk = peaks()
    for name in per_op:
        per_op[name]["frac"] = round(per_op[name]["GB/s"] / pk["hbm_gbs"], 4)
        per_op[name]["frac_of_nominal"] = round(per_op[name]["GB/s"] / NOMINAL_HBM_GBS, 4)
    dom = max(per_op, key=lambda n: per_op[n]["ms"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": per_op[dom]["GB/s"], "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": per_op[dom]["frac"],
                "peak_source": f"{pk['source']} hbm_gbs (of {pk['source']})",
                "frac_of_nominal": per_op[dom]["frac_of_nominal"], "nominal_peak": NOMINAL_HBM_GBS,
                "traffic": traffic_for(dom)}

    # the same step with the scan on a second stream (the three ops are
    # independent): its look-back waits overlap the other two ops' streaming.
    # Reported beside the sequential step, whose per-kernel times give the
    # roofline; here the kernels share HBM, so only the step time is meaningful.
    concurrent = None
    if len(ops) == 3 and not args.no_extras:
        concurrent = run_step_concurrent(torch, D, dev, stream, op_reduce, op_scan, op_transpose, K,
                                         args.warmup, step_bytes, pk["hbm_gbs"])

    # end to end: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, torch, dev, stream, ops, nb, Rn, Sn, T, op_reduce, op_scan, op_transpose, world)

    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + (" (small)" if args.small else ""),
                       "reduce_n": Rn, "scan_n": Sn, "transpose": [T, T],
                       "reduce_view": "group(1024)[[block]].group(32)[[warp]][[thread]]",
                       "l2": "inputs larger than L2 (129 MB); no flush", "parallelism": f"replicas x{world}",
                       "schedules": schedules, "general_kernels": bool(args.generic)},
            "ops": per_op, "roofline": roofline, "gpu_launches": K * len(ops), "e2e": e2e}
    if concurrent:
        line["step_concurrent"] = concurrent
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if not args.no_extras and not args.small:
        line["matmul"] = run_matmul(torch, D, dev, stream, pk)
        line["segmented"] = run_segmented(torch, D, synth, dev, stream)
        line["view_overhead"] = run_view_overhead(torch, D, synth, dev, stream)
        line["split_launch"] = run_split_launch(torch, D, synth, dev)
        line["operators"] = run_operators(torch, D, dev, stream, xr, xs, pk)
        if not args.no_model:
            line["schedule_model"] = run_schedule_model(torch, D, synth)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sz, only)
    return line


def autotune_step(D, stream, probs, names):
    """Exhaustive autotuning of the step's own problems (every schedule
    candidate timed with CUDA events on the step's buffers); the fastest is
    recorded and used by the timed step.  Returns {op: {chosen, us: [...]}}."""
    import ctypes
    out = {}
    for name in names:
        op, dt, n, aux, x, y, ws, view = probs[name]
        p = D.make_problem(op, dt, n, aux, **(view or {}))
        b = D.TuneBuffers()
        b.inp, b.out, b.sums, b.offsets = x.data_ptr(), y.data_ptr(), None, None
        b.ws, b.ws_bytes = ws.data_ptr(), ws.numel()
        nc = D.candidate_count(op)
        us = (ctypes.c_float * nc)()
        D._check(D.lib().desc_tune_measure(p.ref(), ctypes.byref(b), 5, D._stream(stream), us),
                 "desc_tune_measure")
        us = list(us)
        best = min(range(nc), key=lambda c: (us[c], c))
        D.desc_tune_record(p, best)
        out[name] = {"chosen": best, "us": [round(u, 1) for u in us]}
    return out


def run_step_concurrent(torch, D, dev, stream, op_reduce, op_scan, op_transpose, K, warmup, step_bytes, peak):
    """The step with the scan on a second stream, forked from and joined back
    to the timing stream every step: reduce then transpose on one stream, the
    scan beside them.  Timed by CUDA events on the timing stream."""
    side = torch.cuda.Stream(dev)

    def step():
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        op_scan(stream=side)
        op_reduce()
        op_transpose()
        join = torch.cuda.Event()
        join.record(side)
        stream.wait_event(join)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if D.desc_stream_status(stream) != 0 or D.desc_stream_status(side) != 0:
        raise RuntimeError("device status after the concurrent step")
    ms = e0.elapsed_time(e1) / K
    gbs = step_bytes / (ms * 1e-3) / 1e9
    return {"ms_per_step": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_copy_peak": round(gbs / peak, 4),
            "steps": K, "schedule": "scan on a second stream beside reduce -> transpose, forked and joined "
                                    "every step"}


def bucket_of(prob):
    """The tuned-table bucket a problem falls in (op, dtype, floor(log2 n),
    floor(log2(aux + 1))), with n and aux as the op call sees them."""
    n, aux = prob["n"], prob["aux"]
    if prob.get("view") is not None:
        if prob["op"] == 1:
            ops = prob["view"][1]
            n = n - sum(o[1] for o in ops if o[0] == "split_snd")
            aux = 0
        elif prob["level"] == 0:
            aux = 0
        else:
            aux = prob["grid"][0]
    elif prob["op"] == 1:
        aux = 0
    elif prob["op"] == 0 and aux <= 1:
        aux = 0
    return (prob["op"], prob["dtype"], max(int(n), 1).bit_length() - 1, (int(aux) + 1).bit_length() - 1)


def regret_study(D, train_probs, test_probs, arena, model, epochs=300, batch=128, lr=2e-3, reps=5, retime_reps=20):
    """Learned schedules against exhaustive autotuning.  Every candidate of
    every problem is timed (training rows, and the held-out ground truth); the
    cost model is trained on the GPU by the library's kernels (log time); on
    each held-out problem the exhaustive winner, the model's pick and the
    default (candidate 0) are then timed again together, in interleaved rounds
    of `retime_reps`, and regret = t(pick) / min(t(winner), t(pick)) - 1 comes
    from those times (so a pick measured as fast as the winner has no regret).
    Also reports how many held-out problems share a tuned-table bucket or an
    exact shape with a training problem."""
    import math
    import time as _time
    import torch
    X, t = [], []
    t0 = _time.time()
    for prob in train_probs:
        us = D.desc_tune_measure(prob, arena, reps)
        for c, row in enumerate(D.feature_rows(prob)):
            X.append(row)
            t.append(math.log(max(us[c], 1e-3)))
    measure_train_s = _time.time() - t0
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    perm = torch.randperm(Xt.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    t1 = _time.time()
    loss = model.train(Xt[perm].contiguous(), tt[perm].contiguous(), epochs, batch, lr)
    torch.cuda.synchronize()
    train_s = _time.time() - t1
    train_buckets = {bucket_of(p) for p in train_probs}

    def shape_key(p):
        L = p.get("lengths")
        return (p["op"], p["dtype"], p["n"], p["aux"], p.get("k", 0), repr(p.get("view")), p.get("level", 0),
                None if L is None else tuple(L.tolist()))
    train_shapes = {shape_key(p) for p in train_probs}
    reg_model, reg_default, exact, exh_s, pick_s, retime_s = [], [], 0, 0.0, 0.0, 0.0
    bucket_overlap = sum(1 for p in test_probs if bucket_of(p) in train_buckets)
    shape_overlap = sum(1 for p in test_probs if shape_key(p) in train_shapes)
    for prob in test_probs:
        a = _time.time()
        us = D.desc_tune_measure(prob, arena, reps)
        exh_s += _time.time() - a
        win = min(range(len(us)), key=lambda c: (us[c], c))
        rows = torch.tensor(D.feature_rows(prob), dtype=torch.float32, device="cuda")
        a = _time.time()
        c, _ = model.pick(rows)
        pick_s += _time.time() - a
        cands = sorted({win, c, 0})
        a = _time.time()
        ut = dict(zip(cands, D.desc_tune_measure_cands(prob, arena, cands, retime_reps)))
        retime_s += _time.time() - a
        best = min(ut[win], ut[c])
        reg_model.append(ut[c] / best - 1.0)
        reg_default.append(ut[0] / min(ut[win], ut[0]) - 1.0)
        exact += int(c == win)
    n = len(test_probs)
    srt = sorted(reg_model)
    return {"train_rows": len(X), "train_problems": len(train_probs), "test_problems": n, "final_loss": loss,
            "mean_regret": sum(reg_model) / n, "p90_regret": srt[int(0.9 * (n - 1))],
            "default_mean_regret": sum(reg_default) / n, "exact_picks": exact / n,
            "overlap": {"bucket": bucket_overlap, "shape": shape_overlap},
            "split": "train: floor(log2 n) even; held out: odd (no shared tuned-table bucket)",
            "retime_reps": retime_reps, "measure_train_s": measure_train_s, "train_s": train_s,
            "exhaustive_test_s": exh_s, "retime_test_s": retime_s, "model_pick_s": pick_s}


def run_schedule_model(torch, D, synth, n_train=860, n_test=500):
    """Learned schedules: exhaustive timings of every candidate of seeded
    problems from the reduce / scan / transpose / segmented / matmul families
    (about 3,000 training rows, sizes with even floor(log2 n)), the cost model
    trained on the GPU by the library's kernels, and its picks on 500 held-out
    problems (odd floor(log2 n): no tuned-table bucket in common) compared with
    the exhaustive tuner and with the default (regret = t(pick) / t(best) - 1,
    from re-timed winners and picks)."""
    arena = D.TuneArena(1 << 27, 5000, max_mm=4096)
    train = synth.tune_problems(n_train, seed=101, part="even")
    test = synth.tune_problems(n_test, seed=202, part="odd")
    model = D.CostModel(synth.mlp_init(D.NUM_FEATURES, 64, seed=303))
    r = regret_study(D, train, test, arena, model, epochs=300, batch=128, lr=2e-3, reps=5)
    del arena
    torch.cuda.empty_cache()
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}


def _time(torch, stream, fn, reps):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_matmul(torch, D, dev, stream, pk, n=8192, forms=("split3", "bf16", "fp32_simt"), quick=False):
    """C = A B at M = N = K = 8192, FP32 N(0,1) inputs: time of one call
    (split pass included), effective TFLOP/s (2 n^3 / t), tensor TFLOP/s
    (products x 2 n^3 / t) against the dense BF16 peak, and the relative
    Frobenius error on 64 sampled rows against an FP64 product (torch, CPU)."""
    import ctypes
    import synth
    A = synth.normal_f32(n * n, seed=1, stream=1, device=dev).reshape(n, n)
    B = synth.normal_f32(n * n, seed=1, stream=2, device=dev).reshape(n, n)
    rows = torch.arange(0, n, n // 64)
    ref = (A[rows].double().cpu() @ B.double().cpu())
    C = torch.empty(n, n, device=dev)
    out = {"shape": [n, n, n], "peak_bf16_tflops": pk["bf16_tflops"],
           "peak_source": f"bf16_tflops (burst, of {pk['source']})"}
    for name, p, nprod, reps in (("split3", D.MM_SPLIT3, 6, 5), ("bf16", D.MM_BF16, 1, 10),
                                 ("fp32_simt", D.MM_FP32_SIMT, 1, 2)):
        if name not in forms:
            continue
        if quick:
            reps = 1
        nb = ctypes.c_size_t(0)
        D.lib().desc_matmul_workspace_size(n, n, n, p, ctypes.byref(nb))
        ws = torch.empty(max(nb.value, 1), dtype=torch.uint8, device=dev)
        ms = _time(torch, stream, lambda: D.desc_matmul(A, B, p, out=C, ws=ws, stream=stream), reps)
        # the same call back to back for about 0.4 s, with the SM clock sampled
        ms_long, clk = ms, None
        if not quick and p != D.MM_FP32_SIMT:
            ck = Clocks(_gpu_uuid(torch, dev))
            ck.start()
            time.sleep(0.2)
            t0 = time.time()
            ms_long = _time(torch, stream, lambda: D.desc_matmul(A, B, p, out=C, ws=ws, stream=stream),
                            max(reps, int(400 / max(ms, 1e-3))))
            t1 = time.time()
            clk = ck.stop(t0, t1)
        got = C[rows].double().cpu()
        err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        eff = 2 * n ** 3 / (ms * 1e-3) / 1e12
        r = {"ms": round(ms, 4), "effective_tflops": round(eff, 1), "rel_frobenius_err": float(f"{err:.3e}")}
        if p != D.MM_FP32_SIMT:
            eff_long = 2 * n ** 3 / (ms_long * 1e-3) / 1e12
            r["sustained"] = {"ms": round(ms_long, 4), "tensor_tflops": round(nprod * eff_long, 1),
                              "frac_of_bf16_sustained_peak": round(nprod * eff_long / pk["bf16_tflops_sustained"], 4)}
            if clk:
                r["sustained"]["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
                # the nominal dense peak at the SM clock the loop ran at
                nom = NOMINAL_BF16_TFLOPS * clk["sm_mhz"] / NOMINAL_SM_MHZ
                r["sustained"]["frac_of_nominal_at_sampled_clock"] = round(nprod * eff_long / nom, 4)
        if p != D.MM_FP32_SIMT:
            r["tensor_tflops"] = round(nprod * eff, 1)
            r["frac_of_bf16_peak"] = round(nprod * eff / pk["bf16_tflops"], 4)
            r["frac_of_nominal_bf16"] = round(nprod * eff / NOMINAL_BF16_TFLOPS, 4)
        out[name] = r
        del ws
    if D.desc_stream_status(stream) != 0:
        raise RuntimeError("device status after matmul")
    return out


def run_view_overhead(torch, D, synth, dev, stream, reps=100, mbs=(256, 512, 1024)):
    """Section 5's overhead experiment on this GPU: each op through its view,
    once with the hand-indexed kernel the lowering selects and once through
    the general kernels that evaluate the lowered affine map element by
    element (desc_force_generic).  Sizes are input bytes (256 MB, 512 MB,
    1 GB); each time is the median of `reps` launches (CUDA events)."""
    import ctypes
    V = D

    def med(fn):
        fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        d = sorted(a.elapsed_time(b) for a, b in ev)
        return d[len(d) // 2]

    def ws_of(query):
        n = ctypes.c_size_t(0)
        query(ctypes.byref(n))
        return torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)

    red_ops = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
               ("select", V.THREAD, V.X)]
    out = {"reps": reps, "sizes": "input bytes", "views": {
        "reduce": "int32, group(1024)[[block]].group(32)[[warp]][[thread]] -> one scalar",
        "scan": "FP32 inclusive scan of the whole array",
        "transpose": "FP32 R x C -> C x R, transpose view on the input"}}
    L = D.lib()
    for mb in mbs:
        n = mb * (1 << 20) // 4
        row = {}
        x = synth.ints_pm1000(n, seed=11, device=dev)
        r = torch.empty(1, dtype=torch.int32, device=dev)
        grid, block = (n // 1024, 1, 1), (1024, 1, 1)
        t = {}
        for gen in (False, True):
            D.desc_force_generic(gen)
            ws = ws_of(lambda b: L.desc_reduce_workspace_size(ctypes.byref(D.make_view([n], red_ops)),
                                                              ctypes.byref(D.make_exec(grid, block)), V.GRID,
                                                              V.I32, b))
            t[gen] = med(lambda: D.desc_reduce(x, [n], red_ops, V.GRID, grid, block, out=r, ws=ws, stream=stream))
            del ws
        D.desc_force_generic(False)
        row["reduce"] = t
        del x
        xs = synth.uniform_grid(n, seed=12, device=dev)
        ys = torch.empty_like(xs)
        t = {}
        for gen in (False, True):
            D.desc_force_generic(gen)
            ws = ws_of(lambda b: L.desc_scan_workspace_size(ctypes.byref(D.make_view([n], [])), None, V.GRID,
                                                            V.F32, b))
            t[gen] = med(lambda: D.desc_scan(xs, [n], [], V.GRID, out=ys, ws=ws, stream=stream))
            del ws
        D.desc_force_generic(False)
        row["scan"] = t
        del xs, ys
        R = 1 << ((n.bit_length() - 1) // 2)
        C = n // R
        xt = synth.normal_f32(n, seed=13, device=dev).reshape(R, C)
        yt = torch.empty(C, R, device=dev)
        t = {}
        for gen in (False, True):
            D.desc_force_generic(gen)
            t[gen] = med(lambda: D.desc_transpose(xt, [R, C], [("transpose", 0)], yt, [C, R], [], stream=stream))
        D.desc_force_generic(False)
        row["transpose"] = t
        del xt, yt
        out[f"{mb}MB"] = {k: {"hand_indexed_ms": round(v[False], 4), "generic_ms": round(v[True], 4),
                              "overhead_pct": round(100 * (v[True] / v[False] - 1), 1)} for k, v in row.items()}
    if D.desc_stream_status(stream) != 0:
        raise RuntimeError("device status after the view-overhead runs")
    return out


def run_operators(torch, D, dev, stream, xr, xs, pk, reps=10):
    """The operators beyond the sum at full size: int32 reduce of 2^30
    values and FP32 / int32 scans of 2^28 values with each operator family
    (maximum, product, xor, arg-maximum; the arg-maximum and the sum also through a reversed view), and FP32 sum scans segmented per
    block of the view group(m)[[block]] (m = 1024, 2^20), CUDA-event means of `reps` calls,
    GB/s of algorithmic bytes (reduce 4 B, scan 8 B per element) and the
    fraction of the measured copy peak."""
    V = D
    Rn, Sn = xr.numel(), xs.numel()
    out = {}
    r_out = torch.empty(1, dtype=torch.int32, device=dev)
    s_out = torch.empty(Sn, dtype=torch.int32, device=dev)
    xsi = xs.view(torch.int32)                         # the same bytes as int32 for the bitwise scans
    import ctypes
    def ws_reduce(n, dt):
        b = ctypes.c_size_t(0)
        D.lib().desc_reduce_workspace_size(ctypes.byref(D.make_view([n], [])), None, V.GRID, dt, ctypes.byref(b))
        return torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
    def ws_scan(n, dt):
        b = ctypes.c_size_t(0)
        D.lib().desc_scan_workspace_size(ctypes.byref(D.make_view([n], [])), None, V.GRID, dt, ctypes.byref(b))
        return torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
    wr, ws_ = ws_reduce(Rn, V.I32), ws_scan(Sn, V.F32)
    for name, flag in (("max", D.MAX), ("prod", D.PROD), ("xor", D.XOR), ("argmax", D.ARGMAX)):
        ms = _time(torch, stream, lambda: D.desc_reduce(xr, [Rn], [], V.GRID, out=r_out, ws=wr, flags=flag,
                                                         stream=stream), reps)
        gbs = 4 * Rn / (ms * 1e-3) / 1e9
        out[f"reduce_i32_{name}"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}
    for name, x, flag in (("f32_max", xs, D.MAX), ("f32_prod", xs, D.PROD), ("i32_xor", xsi, D.XOR),
                          ("f32_argmax", xs, D.ARGMAX)):
        o = s_out if flag in (D.XOR, D.ARGMAX) else s_out.view(torch.float32)
        ms = _time(torch, stream, lambda: D.desc_scan(x, [Sn], [], V.GRID, out=o, ws=ws_, flags=flag,
                                                       stream=stream), reps)
        gbs = 8 * Sn / (ms * 1e-3) / 1e9
        out[f"scan_{name}"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}
    # the arg-maximum scan through a reversed view (a map of one dim, stride -1)
    ms = _time(torch, stream, lambda: D.desc_scan(xs, [Sn], [("reverse", 0)], V.GRID, out=s_out, ws=ws_, flags=D.ARGMAX,
                                                   stream=stream), reps)
    gbs = 8 * Sn / (ms * 1e-3) / 1e9
    out["scan_f32_argmax_reversed"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}
    ms = _time(torch, stream, lambda: D.desc_scan(xs, [Sn], [("reverse", 0)], V.GRID, out=s_out.view(torch.float32),
                                                   ws=ws_, stream=stream), reps)
    gbs = 8 * Sn / (ms * 1e-3) / 1e9
    out["scan_f32_sum_reversed"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}
    # segmented per level: group(m)[[block]], one segment per block of the view
    so = s_out.view(torch.float32)
    for m in (1024, 1 << 20):
        ops = [("group", m, 0), ("select", V.BLOCK, V.X)]
        ms = _time(torch, stream, lambda: D.desc_scan(xs, [Sn], ops, V.BLOCK, (Sn // m, 1, 1), (1, 1, 1), out=so,
                                                       ws=ws_, stream=stream), reps)
        gbs = 8 * Sn / (ms * 1e-3) / 1e9
        out[f"scan_f32_sum_per_block_{m}"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1),
                                              "frac": round(gbs / pk["hbm_gbs"], 4)}
    if D.desc_stream_status(stream) != 0:
        raise RuntimeError("device status after the operators")
    del s_out, wr, ws_
    return out


def run_sanitize_case(torch, D, synth, dev):
    """One small call of every memory-bound kernel (for a race checker):
    reduce through the hierarchical view and a general map, the look-back
    scan (plain, per-block segments, mapped, CSR), the map scan (arg
    operator), the per-segment group schedules, the tiled transpose, the
    tiled general copy and the element-wise copy.  Returns the call names."""
    V = D
    n = 1 << 16
    x = synth.ints_pm1000(n, seed=1, device=dev)
    xf = synth.uniform_grid(n, seed=2, device=dev)
    hier = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
            ("select", V.THREAD, V.X)]
    calls = []
    D.desc_reduce(x, [n], hier, V.BLOCK, (n // 1024, 1, 1), (1024, 1, 1)); calls.append("reduce runs")
    D.desc_reduce(x, [256, 256], [("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (256, 1, 1), (1, 1, 1))
    calls.append("reduce affine")
    D.desc_scan(xf, [n], [], V.GRID); calls.append("scan")
    D.desc_scan(x, [n], [("group", 4096, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (16, 1, 1), (1, 1, 1))
    calls.append("scan per block")
    D.desc_scan(xf, [n], [("reverse", 0)], V.GRID); calls.append("scan mapped")
    D.desc_scan(x, [n], [], V.GRID, flags=D.ARGMAX); calls.append("map scan (argmax)")
    L = synth.loguniform_lengths(100, seed=3, max_len=2000, device=dev)
    off = synth.offsets_from_lengths(L)
    xs = synth.uniform_grid(int(off[-1]), seed=4, device=dev)
    D.desc_segmented_reduce_scan(xs, off); calls.append("segmented tiles")
    for c in (3, 4):
        D.desc_force_candidate(D.OP_SEGMENTED, c)
        D.desc_segmented_reduce_scan(xs, off); calls.append(f"segmented group {c}")
    D.desc_force_candidate(D.OP_SEGMENTED, -1)
    t = synth.normal_f32(300 * 500, seed=5, device=dev).reshape(300, 500)
    D.desc_transpose(t, [300, 500], [("transpose", 0)], torch.empty(500, 300, device=dev), [500, 300], [])
    calls.append("transpose")
    c3 = synth.normal_f32(6 * 40 * 48, seed=6, device=dev).reshape(6, 40, 48)
    D.desc_transpose(c3, [6, 40, 48], [("transpose", 0), ("transpose", 1)], torch.empty(40, 48, 6, device=dev),
                     [40, 48, 6], []); calls.append("general copy (tiled)")
    D.desc_transpose(t, [300, 500], [("reverse", 1), ("transpose", 0)], torch.empty(500, 300, device=dev),
                     [500, 300], []); calls.append("general copy")
    torch.cuda.synchronize()
    if D.desc_stream_status() != 0:
        raise RuntimeError("device status after the sanitizer case")
    return calls


def run_split_launch(torch, D, synth, dev, iters=20, replays=10):
    """One launch whose first blocks reduce and whose other blocks transpose
    (desc_split_reduce_transpose) against the two separate launches, both
    captured in CUDA graphs (so host time does not enter), per iteration:
    small (int32 reduce of 2^20, 1024^2 transpose) and large (2^28, 8192^2)."""
    import ctypes
    res = {}
    D.desc_force_candidate(D.OP_REDUCE, 0)              # the schedule the split launch runs
    try:
        for name, n, T in (("small", 1 << 20, 1024), ("large", 1 << 28, 8192)):
            x = synth.ints_pm1000(n, seed=21, device=dev)
            t = synth.normal_f32(T * T, seed=22, device=dev).reshape(T, T)
            to = torch.empty(T, T, device=dev)
            r = torch.empty(1, dtype=torch.int32, device=dev)
            nb = ctypes.c_size_t(0)
            D.lib().desc_reduce_workspace_size(ctypes.byref(D.make_view([n], [])), None, D.GRID, D.I32,
                                               ctypes.byref(nb))
            ws = torch.empty(max(nb.value, 1), dtype=torch.uint8, device=dev)
            side = torch.cuda.Stream(dev)

            def sep(st):
                D.desc_reduce(x, [n], [], D.GRID, out=r, ws=ws, stream=st)
                D.desc_transpose(t, [T, T], [("transpose", 0)], to, [T, T], [], stream=st)

            def fused(st):
                D.desc_split_reduce_transpose(x, [n], [], D.GRID, None, None, t, to, out=r, ws=ws, stream=st)

            times = {}
            for key, fn in (("separate", sep), ("split", fused)):
                with torch.cuda.stream(side):
                    fn(side)                              # warm-up outside the capture
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=side):
                    for _ in range(iters):
                        fn(side)
                g.replay()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(replays):
                    g.replay()
                b.record()
                torch.cuda.synchronize()
                times[key] = a.elapsed_time(b) / (replays * iters)
            total = int(x.to(torch.int64).sum().item())
            if int(r.item()) != ((total + (1 << 31)) % (1 << 32)) - (1 << 31):   # int32 wrap-around
                raise RuntimeError("split launch reduce result")
            res[name] = {"reduce_n": n, "transpose": [T, T], "separate_us": round(1000 * times["separate"], 2),
                         "split_us": round(1000 * times["split"], 2),
                         "speedup": round(times["separate"] / times["split"], 3)}
            del x, t, to, ws
    finally:
        D.desc_force_candidate(D.OP_REDUCE, -1)
    return res


def segment_schedules(D, stream, x, off, out, sums, ws, reps=5):
    """Every schedule of the batched call timed on these buffers (CUDA-event
    medians, desc_tune_measure): microseconds per candidate."""
    import ctypes
    nseg = off.numel() - 1
    p = D.make_problem(D.OP_SEGMENTED, D.F32, x.numel(), nseg, off[1:].cpu() - off[:-1].cpu())
    b = D.TuneBuffers()
    b.inp, b.out, b.sums, b.offsets = x.data_ptr(), out.data_ptr(), sums.data_ptr(), off.data_ptr()
    b.ws, b.ws_bytes = ws.data_ptr(), ws.numel()
    nc = D.candidate_count(D.OP_SEGMENTED)
    us = (ctypes.c_float * nc)()
    D._check(D.lib().desc_tune_measure(p.ref(), ctypes.byref(b), reps, D._stream(stream), us), "desc_tune_measure")
    names = ["tiles 16384", "tiles 8192", "tiles 4096", "warp per segment", "CTA per segment"]
    return {names[c]: round(us[c], 1) for c in range(nc)}


def run_segmented(torch, D, synth, dev, stream, nseg=20000):
    """20,000 FP32 segments, lengths log-uniform in [1, 2^20]: every segment
    reduced and inclusive-scanned.  One graph-captured persistent launch vs.
    the same call launched directly vs. one scan + one reduce launch per
    segment.  GB/s counts 8 B per element + 8 B of offsets + 4 B per sum.
    Also every schedule of the call (tiles of three sizes, a warp or a CTA
    per segment) on this workload and on 2,000,000 segments of at most 256
    points, where a group of threads per segment pays."""
    L = synth.loguniform_lengths(nseg, seed=7, device=dev)
    off = synth.offsets_from_lengths(L)
    total = int(off[-1])
    x = synth.uniform_grid(total, seed=8, device=dev)
    out = torch.empty_like(x)
    sums = torch.empty(nseg, device=dev)
    ws = D.desc_segmented_workspace(nseg, total, dev)
    g = D.SegmentedGraph(x, off, out, sums, ws)
    t_graph = _time(torch, stream, lambda: g.launch(stream), 10)
    t_direct = _time(torch, stream, lambda: D.desc_segmented_reduce_scan(x, off, out=out, sums=sums, ws=ws,
                                                                        stream=stream), 10)
    h = off.cpu().tolist()
    t_per = _time(torch, stream, lambda: D.desc_segmented_reduce_scan_per_segment(x, h, out=out, sums=sums, ws=ws,
                                                                                 stream=stream), 1)
    g.close()
    sched = segment_schedules(D, stream, x, off, out, sums, ws)
    del x, out, sums, ws, g
    nbytes = 8 * total + 8 * (nseg + 1) + 4 * nseg
    # many short segments
    ns2 = 2_000_000
    L2 = synth.loguniform_lengths(ns2, seed=9, max_len=256, device=dev)
    off2 = synth.offsets_from_lengths(L2)
    tot2 = int(off2[-1])
    x2 = synth.uniform_grid(tot2, seed=10, device=dev)
    o2 = torch.empty_like(x2)
    s2 = torch.empty(ns2, device=dev)
    ws2 = D.desc_segmented_workspace(ns2, tot2, dev)
    sched_short = segment_schedules(D, stream, x2, off2, o2, s2, ws2)
    b2 = 8 * tot2 + 8 * (ns2 + 1) + 4 * ns2
    best2 = min(sched_short.values())
    del x2, o2, s2, ws2
    if D.desc_stream_status(stream) != 0:
        raise RuntimeError("device status after segmented")
    return {"segments": nseg, "elements": total, "graph_ms": round(t_graph, 4), "direct_ms": round(t_direct, 4),
            "per_segment_ms": round(t_per, 3), "graph_GB/s": round(nbytes / (t_graph * 1e-3) / 1e9, 1),
            "frac_of_nominal": round(nbytes / (t_graph * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
            "speedup_vs_per_segment": round(t_per / t_graph, 1), "schedules_us": sched,
            "short_segments": {"segments": ns2, "elements": tot2, "max_len": 256, "schedules_us": sched_short,
                               "best_GB/s": round(b2 / (best2 * 1e-6) / 1e9, 1)}}


def run_e2e(args, torch, dev, stream, ops, nb, Rn, Sn, T, op_reduce, op_scan, op_transpose, world):
    """The step end to end through the public API: every step copies its
    inputs from pinned host memory and its results back.  Three streams -- one
    for host-to-device copies, one for the ops, one for device-to-host copies
    -- with double-buffered device inputs and outputs, so an op runs while the
    next op's input travels in and the previous results travel back (the link
    carries both directions at once).  Events order each buffer's reuse."""
    import synth
    names = [n for n, _ in ops]
    h = {}
    if "reduce" in names:
        h["xr"] = torch.empty(Rn, dtype=torch.int32, pin_memory=True)
        h["or"] = torch.empty(1, dtype=torch.int32, pin_memory=True)
        h["xr"].copy_(synth.ints_pm1000(Rn, seed=1, device=dev))
    if "scan" in names:
        h["xs"] = torch.empty(Sn, dtype=torch.float32, pin_memory=True)
        h["os"] = torch.empty(Sn, dtype=torch.float32, pin_memory=True)
        h["xs"].copy_(synth.uniform_grid(Sn, seed=2, device=dev))
    if "transpose" in names:
        h["xt"] = torch.empty(T, T, dtype=torch.float32, pin_memory=True)
        h["ot"] = torch.empty(T, T, dtype=torch.float32, pin_memory=True)
        h["xt"].copy_(synth.normal_f32(T * T, seed=3, device=dev).reshape(T, T))
    two = lambda f: [f() for _ in range(2)]
    dr = two(lambda: torch.empty(Rn, dtype=torch.int32, device=dev)) if "reduce" in names else None
    ds = two(lambda: torch.empty(Sn, dtype=torch.float32, device=dev)) if "scan" in names else None
    dt_ = two(lambda: torch.empty(T, T, dtype=torch.float32, device=dev)) if "transpose" in names else None
    or_ = two(lambda: torch.empty(1, dtype=torch.int32, device=dev))
    os_ = two(lambda: torch.empty(Sn, dtype=torch.float32, device=dev)) if ds is not None else None
    ot = two(lambda: torch.empty(T, T, dtype=torch.float32, device=dev)) if dt_ is not None else None
    sin, sk, sout = torch.cuda.Stream(dev), stream, torch.cuda.Stream(dev)
    ev = lambda: [torch.cuda.Event() for _ in range(2)]
    loaded = {k: ev() for k in ("r", "s", "t")}        # input of buffer b is on the device
    ready = {k: ev() for k in ("r", "s", "t")}         # output of buffer b is computed
    consumed, shipped = ev(), ev()                     # buffer b's inputs read / outputs copied back
    used = [False, False]
    h2d = d2h = 0

    def step(k):
        nonlocal h2d, d2h
        b = k % 2
        h2d = d2h = 0
        plan = []
        if dr is not None:
            plan.append(("r", h["xr"], dr[b], Rn * 4, lambda: op_reduce(dr[b], or_[b]), h["or"], or_[b], 4))
        if ds is not None:
            plan.append(("s", h["xs"], ds[b], Sn * 4, lambda: op_scan(ds[b], os_[b], stream=sk), h["os"], os_[b],
                         Sn * 4))
        if dt_ is not None:
            plan.append(("t", h["xt"], dt_[b], T * T * 4, lambda: op_transpose(dt_[b], ot[b]), h["ot"], ot[b],
                         T * T * 4))
        with torch.cuda.stream(sin):
            if used[b]:
                sin.wait_event(consumed[b])             # the ops of step k - 2 have read buffer b
            for key, hx, dx, nbytes, _, _, _, _ in plan:
                dx.copy_(hx, non_blocking=True)
                h2d += nbytes
                loaded[key][b].record(sin)
        with torch.cuda.stream(sk):
            if used[b]:
                sk.wait_event(shipped[b])               # step k - 2's results have left buffer b
            for key, _, _, _, op, _, _, _ in plan:
                sk.wait_event(loaded[key][b])
                op()
                ready[key][b].record(sk)
            consumed[b].record(sk)
        with torch.cuda.stream(sout):
            for key, _, _, _, _, ho, do, nbytes in plan:
                sout.wait_event(ready[key][b])
                ho.copy_(do, non_blocking=True)
                d2h += nbytes
            shipped[b].record(sout)
        used[b] = True

    K = max(3, min(args.steps, args.e2e_steps))
    for k in range(2):
        step(k)
    torch.cuda.synchronize(dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(sk)
    for k in range(K):
        step(k)
    sk.wait_stream(sin)
    sk.wait_stream(sout)
    e.record(sk)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(e)
    if world > 1:
        ms = max_over_ranks(torch, ms, dev)
    step_bytes = sum(nb[n] for n in names)
    return {"value": round(job_rate(world, step_bytes, K, ms), 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": K,
            "ms_per_step": round(ms / K, 3),
            "overlap": "three streams: inputs in, ops, results out; double-buffered device inputs and outputs"}


# --------------------------------------------------------------------- oracle
ORACLE_SCALE = 1.0          # the oracle's sample: reduce 2^26, scan 2^24, transpose 4096^2 (both CPU legs)


def oracle_samples(sz, only, scale=ORACLE_SCALE):
    """Seeded inputs of the CPU oracle's bounded sample of the workload."""
    import synth
    nr = max(1 << 12, int((1 << 26) * scale))
    ns = max(1 << 12, int((1 << 24) * scale))
    tt = max(64, int(4096 * scale ** 0.5))
    out = {}
    if not only or "reduce" in only:
        out["reduce"] = synth.ints_pm1000(nr, seed=11).numpy()
    if not only or "scan" in only:
        out["scan"] = synth.uniform_grid(ns, seed=12).numpy()
    if not only or "transpose" in only:
        out["transpose"] = synth.normal_f32(tt * tt, seed=13).numpy().reshape(tt, tt)
    return out


def sample_desc(samples):
    d = {k: (list(v.shape) if k == "transpose" else v.size) for k, v in samples.items()}
    return f"reduce {d.get('reduce')} int32, scan {d.get('scan')} FP32, transpose {d.get('transpose')} FP32"


def oracle_rate(sz, samples):
    """GB/s of the CPU oracle on the samples, weighted by the full step's
    bytes: each op's sample time is scaled to its full size."""
    import numpy as np
    from oracle import ops as O
    full = op_bytes(sz)
    t_est = 0.0
    for op, x in samples.items():
        t = time.perf_counter()
        if op == "reduce":
            O.reduce(x, [x.size], [], 0)
            t_est += (time.perf_counter() - t) * full["reduce"] / (4 * x.size)
        elif op == "scan":
            O.scan(x, np.zeros(x.size, np.float32), [x.size], [], 0)
            t_est += (time.perf_counter() - t) * full["scan"] / (8 * x.size)
        else:
            O.transpose2d(x)
            t_est += (time.perf_counter() - t) * full["transpose"] / (8 * x.size)
    step_bytes = sum(full[k] for k in samples)
    return step_bytes / t_est / 1e9


def _oracle_task(task):
    """One oracle call on one sample (runs in a spawned worker: NumPy and the
    oracle only).  Returns the seconds it took."""
    import numpy as np
    from oracle import ops as O
    op, x = task
    t = time.perf_counter()
    if op == "reduce":
        O.reduce(x, [x.size], [], 0)
    elif op == "scan":
        O.scan(x, np.zeros(x.size, np.float32), [x.size], [], 0)
    else:
        O.transpose2d(x)
    return time.perf_counter() - t


def oracle_rate_all_cores(sz, samples, cores):
    """The oracle as it stands on every host core at once: each worker runs
    its own copy of the same samples (independent problems, weak scaling);
    GB/s = cores x the step-weighted bytes / the slowest worker's time per op."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    full = op_bytes(sz)
    scale = {"reduce": lambda x: full["reduce"] / (4 * x.size), "scan": lambda x: full["scan"] / (8 * x.size),
             "transpose": lambda x: full["transpose"] / (8 * x.size)}
    t_est = 0.0
    # a pool that fails to start raises (BrokenProcessPool) instead of retrying for ever
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        first = next(iter(samples.items()))
        list(pool.map(_oracle_task, [(first[0], first[1][:64])] * cores, timeout=120))   # workers up
        for op, x in samples.items():
            t_est += max(pool.map(_oracle_task, [(op, x)] * cores, timeout=600)) * scale[op](x)
    step_bytes = sum(full[k] for k in samples)
    return cores * step_bytes / t_est / 1e9


def cpu_baseline(sz, only):
    samples = oracle_samples(sz, only)
    v = oracle_rate(sz, samples)
    out = {"value": round(v, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": sample_desc(samples) + " (NumPy, single-threaded; the reference arm's sample); rates "
                     "weighted by the full step's bytes"}
    cores = os.cpu_count() or 1
    if cores > 1:
        try:
            va = oracle_rate_all_cores(sz, samples, cores)
            out["all_cores"] = {"value": round(va, 3), "unit": "GB/s", "cores": cores,
                                "sample": "one copy per core of the same sample (spawned workers)"}
        except Exception as e:                           # no process pool here: the single-core figure stands
            out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args, rank, world):
    """The CPU oracle as it stands, timed on the same bounded sample as the
    default line's cpu_baseline: inputs drawn once, then W untimed and K timed
    passes over the sample, each pass's rate weighted by the full step's bytes."""
    if rank != 0:
        return None
    sz = sizes(args.small)
    only = set(args.ops.split(",")) if args.ops else None
    samples = oracle_samples(sz, only)
    for _ in range(args.warmup):
        oracle_rate(sz, samples)
    t0 = time.perf_counter()
    rates = [oracle_rate(sz, samples) for _ in range(args.steps)]
    el = time.perf_counter() - t0
    value = len(rates) / sum(1.0 / r for r in rates)     # bytes-weighted mean rate
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + (" (small)" if args.small else ""), "reduce_n": sz["reduce_n"],
                       "scan_n": sz["scan_n"], "transpose": [sz["T"], sz["T"]]},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: " + sample_desc(samples) + "; rates weighted by the full step's "
                                       "bytes"},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="small case for profiler captures")
    ap.add_argument("--ops", default="", help="comma list: subset of reduce,scan,transpose")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true", help="skip the matmul and segmented measurements")
    ap.add_argument("--no-model", action="store_true", help="skip the learned-schedule regret study")
    ap.add_argument("--no-tune", action="store_true", help="time the default schedules, without autotuning")
    ap.add_argument("--generic", action="store_true",
                    help="run the step's views through the general kernels (desc_force_generic), for profiles")
    ap.add_argument("--save-tune", default="", help="save the tuned schedule table to this file")
    ap.add_argument("--load-tune", default="", help="use a saved schedule table instead of tuning")
    ap.add_argument("--case", choices=["step", "matmul", "segmented", "overhead", "split", "sanitize", "operators"],
                    default="step",
                    help="matmul / segmented: run only that measurement (for profiler captures)")
    ap.add_argument("--mm-n", type=int, default=8192, help="matmul size for --case matmul")
    ap.add_argument("--mm-prec", default="split3,bf16,fp32_simt",
                    help="matmul forms for --case matmul (comma list of split3, bf16, fp32_simt)")
    ap.add_argument("--mm-quick", action="store_true",
                    help="--case matmul: one warm-up and one timed call per form, no sustained loop")
    ap.add_argument("--seg-count", type=int, default=20000, help="segments for --case segmented")
    args = ap.parse_args()
    if args.warmup < 3 and not args.small:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.case != "step":
        import torch
        import paper_2305_03448_gb300 as D
        import synth
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        if args.case == "matmul":
            line = {"case": "matmul", "matmul": run_matmul(torch, D, dev, stream, peaks(), n=args.mm_n,
                                                           forms=args.mm_prec.split(","), quick=args.mm_quick)}
        elif args.case == "split":
            line = {"case": "split", "split_launch": run_split_launch(torch, D, synth, dev)}
        elif args.case == "overhead":
            line = {"case": "overhead", "view_overhead": run_view_overhead(torch, D, synth, dev, stream)}
        elif args.case == "sanitize":
            line = {"case": "sanitize", "calls": run_sanitize_case(torch, D, synth, dev)}
        elif args.case == "operators":
            sz = sizes(args.small)
            xr = synth.ints_pm1000(sz["reduce_n"], seed=1, device=dev)
            xs = synth.uniform_grid(sz["scan_n"], seed=2, device=dev)
            line = {"case": "operators", "operators": run_operators(torch, D, dev, stream, xr, xs, peaks())}
        else:
            line = {"case": "segmented", "segmented": run_segmented(torch, D, synth, dev, stream, nseg=args.seg_count)}
    else:
        line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
