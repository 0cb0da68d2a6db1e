"""Benchmark: exp(tau L) applies per second on one GB300 (or N replicas).

One step = one application of R(tau L) = sum_m b_m (tau L - alpha_m)^{-1} to
every right-hand side of the workload (both tree sweeps for every distinct
pole plus the pole sum), with operators and state resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle (the
only reference this method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

# The oracle legs below are timed with single-threaded BLAS, so that their stated core
# counts hold (one per process); set before numpy loads.  The GPU leg does no host BLAS.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "exp(tau L) applies/sec at stated rel. L2 error, mixed/batched vs FP64 on 1 GB300"
UNIT = "applies/s"
# FP64 fused multiply-add throughput measured on a GB300 (8 independent
# FMA chains per thread, 1216 blocks x 256 threads, ~1995 MHz): 1.207 TFLOP/s
FP64_PEAK_TFLOPS = 1.207
# FP32 FMA throughput measured the same way: 75.4 TFLOP/s
FP32_PEAK_TFLOPS = 75.4
DEFAULT = W.SW_16X16_P16.name


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"expop_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            t = [x.strip() for x in line.split(",")]
            if len(t) < 8:
                continue
            try:
                sm.append(float(t[0]))
                smax = max(smax, float(t[1]))
            except ValueError:
                continue
            for n, v in zip(names, t[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_operator(eo, w, g, x, y, R, precision, poles=0, dense_leaves=False, fitter="line", root_dense=False,
                   merge_dense=False, tensor_leaves=False, merge_fuse=0):
    # the tensor-core leaf path is a reduced-precision path of the dense leaf operators
    tl = bool(tensor_leaves) and precision == "df32"
    if w.kind == "wave":
        c = W.wave_c(w, x, y)
        if fitter == "gauss":
            # the paper's construction takes the step, not a pole count: the step the
            # line fit chooses for this workload's pole count
            tau = eo.fit(poles or w.n_poles)[2] / W.BAND[w.name]
            return eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], tau=tau, c2=c * c, max_rhs=R,
                               precision=precision, fitter="gauss")
        return eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=poles or w.n_poles, c2=c * c,
                           max_rhs=R, precision=precision, tensor_leaves=tl, merge_fuse=merge_fuse)
    pr = w.params
    # a pole-count override (profiling cases) replaces the fixed step by tau = X(poles) / band
    return eo.Operator(g, eo.SW_WALLS, band=W.BAND[w.name], tau=0.0 if poles else w.tau, n_poles=poles,
                       f=pr["f"], g=pr["g"], H=pr["H"], shared_ops=True, max_rhs=R, precision=precision,
                       dense_leaves=dense_leaves or tl, fitter=fitter, root_dense=root_dense, merge_dense=merge_dense,
                       sw_consistent=bool(pr.get("consistent", False)), tensor_leaves=tl, merge_fuse=merge_fuse)


def is_periodic(w):
    return bool(w.params.get("periodic", False))


def oracle_problem(w, tau, x, y):
    """The oracle's discrete problem of workload w (test infrastructure: the CPU
    baseline legs only)."""
    from oracle import sem
    from oracle.resolvent import Problem
    og = sem.Grid(w.nlx, w.nly, w.p, periodic=is_periodic(w))
    if w.kind == "wave":
        c = W.wave_c(w, x, y)
        return Problem(og, "wave", tau, c2=c * c)
    pr = w.params
    return Problem(og, "sw", tau, f=pr["f"], g=pr["g"], H=pr["H"], consistent=bool(pr.get("consistent", False)))


def timed_steps(torch, op, u, steps, stream, dist, label="timed", trace=False):
    """K steps bracketed by barrier + synchronize, CUDA events on the launching stream.
    The steps sit in an NVTX range (``label``) so that a profiler can select them.
    trace=True turns the library's per-launch tracing on for this pass (CUDA events
    around every launch) and returns its per-class times; the headline number is
    taken with trace=False."""
    if trace:
        op.set_timing(True)
        op.timing()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push(label)
    for _ in range(steps):
        op.apply(u, 1)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    tim = None
    if trace:
        tim = op.timing()
        op.set_timing(False)
    return ms, tim


def plan_levels(nlx, nly, q):
    """Boxes, interface and boundary sizes of every merge level (the library's
    plan: pairs merged alternately along x and y, from the leaves to the root)."""
    sx = sy = 1
    nbx, nby = nlx, nly
    out = []
    d = 0
    while nbx * nby > 1:
        dr = d
        if dr == 0 and nbx == 1:
            dr = 1
        if dr == 1 and nby == 1:
            dr = 0
        d = 1 - dr
        n3 = (sy if dr == 0 else sx) * q
        if dr == 0:
            sx, nbx = 2 * sx, nbx // 2
        else:
            sy, nby = 2 * sy, nby // 2
        out.append({"nbox": nbx * nby, "n3": n3, "nbd": 2 * (sx + sy) * q})
    return out


TC_SLICES, TC_MT, TC_NT, TC_KS = 6, 128, 32, 16


def tensor_flops(w, P, R, shared):
    """bf16 MMA flops the tensor-core leaf down-solve issues in one step: per pole,
    right-hand-side tile (32 columns) and M tile (128 operator rows), every slice pair
    (i + j <= S + 1) of every K step of the X and Y blocks, four real products each."""
    q = w.p - 2
    ni, nb = q * q, 4 * q
    nleaf = w.nlx * w.nly
    tiles = -(-nleaf * R // TC_NT) if shared else nleaf * (-(-R // TC_NT))
    ksteps = -(-ni // TC_KS) + -(-nb // TC_KS)
    pairs = TC_SLICES * (TC_SLICES + 1) // 2
    return float(P) * tiles * 2 * ksteps * pairs * 4 * 2.0 * TC_MT * TC_NT * TC_KS


def class_work(op, w, R, prec, fd, root_c4=False, merge_sym=False, periodic=False):
    """Algorithmic FP64-equivalent flops (8 per complex multiply-add) and bytes
    of one step, per kernel class, with the arithmetic precision of each.
    root_c4: the wall solve runs as four Fourier blocks of a quarter of the wall
    nodes each (square walled domain), a quarter of the dense inverse's entries.
    merge_sym: shared levels apply even/odd blocks (Z in two, U and S in four), which
    every level of an even q has.  periodic: the root solve is the seam system of
    half the root's boundary nodes, and a Dirichlet root keeps its parent blocks."""
    q = w.p - 2
    ni, nb = q * q, 4 * q
    P = int((op.alpha.imag >= 0).sum())
    nleaf = w.nlx * w.nly
    K = 2 if w.kind == "wave" else 3
    shared = w.kind == "sw"
    nlo = 1 if shared else nleaf
    esz = 8 if prec == "fp32" else 16
    n_int = nleaf * ni
    cols = P * nleaf * R
    work = {}
    if fd:
        # per (pole, leaf, rhs): up 4K q^2 (sources) + 32 q^2 (contractions and
        # 1-D transforms); down 32 q^2 (edge transforms, rank-one coupling) + 4K q^2.
        # Arithmetic: FP32 pairs with the FP32-pair precision, FP64 otherwise
        fp = "df32" if prec == "df32" else "fp64"
        work["up_leaf"] = ((4 * K + 32) * ni * cols, cols * nb * 16 + P * K * ni * 16 + R * K * n_int * 8, fp)
        work["down_leaf"] = ((4 * K + 32) * ni * cols, cols * nb * 16 + P * K * ni * 16, fp)
    else:
        work["up_leaf"] = (8.0 * cols * nb * ni, P * nlo * nb * ni * esz + cols * nb * 16 + R * K * n_int * 8, prec)
        work["down_leaf"] = (8.0 * cols * ni * (ni + nb),
                             P * nlo * ni * (ni + nb) * esz + cols * (2 * ni * 8 + nb * 16), prec)
    lv = plan_levels(w.nlx, w.nly, q)
    uf = ub = df = db = 0.0
    for i, l in enumerate(lv):
        root = i == len(lv) - 1
        par = not (root and w.kind == "wave" and not periodic)
        zu = l["n3"] + (l["nbd"] if par else 0)
        nbo = 1 if shared else l["nbox"]
        sym = merge_sym and shared and q % 2 == 0
        # entries of the blocks the apply reads: [-Z; U] and S, or their even/odd blocks
        zent = (l["n3"] // 2) * (l["n3"] + (l["nbd"] // 2 if par else 0)) if sym else zu * l["n3"]
        sent = l["n3"] * l["nbd"] // 4 if sym else l["n3"] * l["nbd"]
        uf += 8.0 * P * l["nbox"] * R * zent
        ub += P * nbo * zent * esz + P * l["nbox"] * R * (2 * l["n3"] + zu) * 16
        if par:
            df += 8.0 * P * l["nbox"] * R * sent
            db += P * nbo * sent * esz + P * l["nbox"] * R * (l["nbd"] + l["n3"]) * 16
    work["up_merge"] = (uf, ub, prec)
    work["down_merge"] = (df, db, prec)
    if periodic:
        nr = lv[-1]["nbd"] // 2
        work["root"] = (8.0 * P * R * nr * nr, P * nr * nr * esz + P * R * 3 * nr * 16, prec)
    elif w.kind == "sw":
        nr = lv[-1]["nbd"]
        ent = 4 * (nr // 4) ** 2 if root_c4 else nr * nr
        work["root"] = (8.0 * P * R * ent, P * ent * esz + P * R * 2 * nr * 16, prec)
    return work


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one step's launches of a
# kernel class, from an ncu capture of the shallow-water workload with 301 poles (151
# distinct), FP32-pair precision, even/odd merge blocks (FP32-pair partial sums and
# boundary data between up levels) and the four-block root.  Traffic grows with the number
# of distinct poles (one block set per pole, read once), so a full step scales it by P / 151.
# Keys: (workload, precision, class).
NCU_TRAFFIC_151 = {
    ("sw_walls_16x16_p16_tau20T", "df32", "up_merge"): 0.4366e9,
    ("sw_walls_16x16_p16_tau20T", "df32", "down_merge"): 0.2942e9,
    ("sw_walls_16x16_p16_tau20T", "df32", "root"): 0.4872e9,
}


def alu_peak(prec):
    # FP32-pair products cost 48 FP32 instructions per complex multiply-add (4
    # split products of 12): pipe bound in FP64-equivalent flops FP32_peak / 2 / 48 * 8
    return {"fp32": FP32_PEAK_TFLOPS, "fp64": FP64_PEAK_TFLOPS, "df32": FP32_PEAK_TFLOPS / 2 / 48 * 8}[prec]


def roofline(op, w, R, tim, prec, pk, pk_kind, fd, root_c4=False, merge_sym=False, periodic=False, tl=False,
             fused=0):
    """Per kernel class: algorithmic work of one step over that class's device
    time per step (CUDA events around its launches), against the ALU peak of
    its arithmetic and the measured HBM copy bandwidth; the class with the
    largest time share is reported as the roofline of the step."""
    work = class_work(op, w, R, prec, fd, root_c4, merge_sym, periodic)
    per = {}
    for cls, (flops, nbytes, pr) in work.items():
        n, ms = tim.get(cls, (0, 0.0))
        if not n:
            continue
        steps = max(1, tim["post_map"][0])
        t = ms / steps / 1e3
        tf = flops / t / 1e12
        gbs = nbytes / t / 1e9
        fa, fh = tf / alu_peak(pr), gbs / pk["hbm_gbs"]
        per[cls] = {"ms_per_step": t * 1e3, "launches_per_step": n / steps, "tflops": tf, "gbs": gbs,
                    "precision": pr, "alu_frac": fa, "hbm_frac": fh, "bound": "alu" if fa >= fh else "hbm"}
    top = max(per, key=lambda c: per[c]["ms_per_step"])
    d = per[top]
    kname = {"up_leaf": "k_fd_up_leaf" if fd else "k_up_leaf", "down_leaf": "k_fd_down_leaf" if fd else "k_down_leaf",
             "up_merge": ("k_up_fused + " if fused else "") + ("k_up_merge_sym" if merge_sym else "k_up_merge"),
             "down_merge": ("k_down_fused + " if fused else "") + ("k_down_merge_sym" if merge_sym else "k_down_merge"),
             "root": "k_root_periodic" if periodic else ("k_root_sw_c4" if root_c4 else "k_root_sw")}[top]
    tname = {"fp32": "float2", "fp64": "double2", "df32": "float4"}[d["precision"]]
    if not (fd and top in ("up_leaf", "down_leaf")):
        kname += "<NC, %s>" % tname
    # headline: algorithmic bytes over time against the measured HBM copy rate; the
    # ALU bound of the class's own arithmetic is reported beside it
    rf = {"bound": "hbm", "achieved": d["gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": d["hbm_frac"],
          "peak_source": pk_kind + " (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)",
          "alu": {"achieved_tflops": d["tflops"], "peak_tflops": alu_peak(d["precision"]),
                  "frac": d["alu_frac"],
                  "unit": "TFLOP/s" + (" (FP64-equivalent)" if d["precision"] == "df32" else ""),
                  "peak_source": {"fp32": "FP32 FMA microbenchmark", "fp64": "FP64 FMA microbenchmark",
                                  "df32": "FP32 FMA microbenchmark / 48 FP32 instructions per FP32-pair complex "
                                          "multiply-add (this algorithm's instruction count, not a chip roof)"}[
                                      d["precision"]]}}
    P = int((op.alpha.imag >= 0).sum())
    if tl and top == "down_leaf":
        # the tensor-core leaf kernel: issued bf16 MMA work against the measured bf16 peak
        # (sustained: the kernel runs inside a long step)
        tf = tensor_flops(w, P, R, shared=(w.kind == "sw")) / (d["ms_per_step"] / 1e3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1900.0))
        rf = {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
              "peak_source": pk_kind + " (MEASURED_PEAKS.json bf16_tflops_sustained, cuBLAS bf16 GEMM)",
              "work": "bf16 tcgen05.mma flops issued (6 slices, 21 slice pairs, 4 real products per "
                      "complex product)", "hbm": {"achieved_gbs": d["gbs"], "frac": d["hbm_frac"]},
              "alu": rf["alu"]}
        kname = "k_tc_down_leaf<6>"
    tr = NCU_TRAFFIC_151.get((w.name, prec, top)) if R == 1 else None
    rf.update({"kernel": kname, "class": top, "traffic": None if tr is None else tr * P / 151 / d["launches_per_step"],
               "traffic_note": None if tr is None else
               "ncu DRAM bytes (read + write) of this class's launches in one step of the 301-pole case, "
               "scaled by P/151, per launch",
               "algorithmic_flops": work[top][0], "algorithmic_bytes": work[top][1],
               "algorithmic_bytes_per_launch": work[top][1] / d["launches_per_step"],
               "avg_launch_ms": d["ms_per_step"] / d["launches_per_step"],
               "launches": tim[top][0], "per_class": per})
    return rf


def run_ours(args):
    import torch
    import paper_1402_5168_gb300 as eo

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    if args.leaves:
        w = W.dataclasses.replace(w, nlx=args.leaves, nly=args.leaves)
    R = args.rhs
    reduced = args.precision != "fp64"
    per = is_periodic(w)
    g = eo.Grid(w.nlx, w.nly, w.p, periodic=per)
    x, y = g.nodes()
    t0 = time.time()
    op = build_operator(eo, w, g, x, y, R, args.precision, args.poles, args.dense_leaves, args.fitter,
                        args.root_dense, args.merge_dense, args.tensor_leaves, args.merge_fuse)
    # the library splits the wall solve of a square walled domain of square leaves into
    # four Fourier blocks unless told not to
    root_c4 = w.kind == "sw" and w.nlx == w.nly and not args.root_dense and not per
    # and applies the even/odd merge blocks on every level of a shared-operator grid
    # (not on periodic grids, nor with the consistent elimination's curl term)
    consistent = bool(w.params.get("consistent", False))
    merge_sym = w.kind == "sw" and not args.merge_dense and not per and not consistent
    tl = bool(args.tensor_leaves) and args.precision == "df32"
    fd = w.kind == "sw" and not args.dense_leaves and not consistent and not tl
    fused = op.fused_levels(R)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    U0 = np.stack([np.stack(W.initial_fields(w, x, y, r)) for r in range(R)])
    u = torch.tensor(U0, device=dev)
    stream = torch.cuda.current_stream()
    clk = Clocks(local) if rank == 0 else None
    for _ in range(args.warmup):
        op.apply(u, 1)
    torch.cuda.synchronize()
    ms, _ = timed_steps(torch, op, u, args.steps, stream, dist)
    clocks = clk.stop() if clk else None
    ms = reduce_max(ms, dist, dev)
    value = world * R * args.steps / (ms / 1e3)
    # a second pass of the same steps with per-launch tracing: kernel classes, shares
    # and the roofline (the headline above ran untraced); the launch sequence of a
    # step is fixed, so the traced pass also counts the launches of the timed one
    ms_traced, tim = timed_steps(torch, op, u, args.steps, stream, dist, label="traced", trace=True)
    launches = sum(v[0] for v in tim.values())
    # end to end through the host entry point: H2D copy, apply, D2H copy each step
    uh_np = torch.tensor(U0).pin_memory().numpy()
    op.apply_host(uh_np, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op.apply_host(uh_np, 1)
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, dev)
    # the FP64 apply of the same workload beside the mixed one: throughput and
    # the mixed path's error after the same number of steps from the same input
    fp64 = None
    if reduced and args.compare_fp64:
        op64 = build_operator(eo, w, g, x, y, R, "fp64", args.poles, args.dense_leaves, args.fitter,
                              args.root_dense, args.merge_dense, merge_fuse=args.merge_fuse)
        u64 = torch.tensor(U0, device=dev)
        for _ in range(args.warmup):
            op64.apply(u64, 1)
        ms64, _ = timed_steps(torch, op64, u64, args.steps, stream, dist, label="timed_fp64")
        a = torch.tensor(U0, device=dev)
        b = torch.tensor(U0, device=dev)
        op.apply(a, 1)
        op64.apply(b, 1)
        err1 = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        half = max(1, args.steps // 2)
        op.apply(a, half - 1)
        op64.apply(b, half - 1)
        n_half = float(torch.linalg.vector_norm(b))
        if args.steps - half:
            op.apply(a, args.steps - half)
            op64.apply(b, args.steps - half)
        err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        growth = float(torch.linalg.vector_norm(b) / torch.linalg.vector_norm(torch.tensor(U0, device=dev)))
        growth_late = float(torch.linalg.vector_norm(b)) / n_half
        # the FP64 trajectory's growth says whether the multi-step comparison measures
        # precision (a bounded trajectory) or rounding amplified by growing discrete modes.
        # The Euclidean norm of a bounded trajectory may still change by a fixed factor
        # (a wave state starting at rest moves energy from u into v), so the test is on
        # the second half of the steps, where growing modes keep growing
        fp64 = {"fp64_value": world * R * args.steps / (ms64 / 1e3), "fp64_ms_per_step": ms64 / args.steps,
                "mixed_vs_fp64_rel_l2_one_step": err1, "mixed_vs_fp64_rel_l2_after_steps": err,
                "mixed_vs_fp64_after_steps": args.steps, "fp64_state_norm_growth": growth,
                "fp64_state_norm_growth_second_half": growth_late,
                "mixed_vs_fp64_after_steps_meaningful": bool(growth_late <= 2.0)}
        del op64
    if rank != 0:
        dist.destroy_process_group()
        return
    pk, pk_kind = peaks()
    ob, wb = op.memory()
    tot_ms = max(sum(t[1] for t in tim.values()), 1e-9)
    fp64 = fp64 or {}
    shares = {k: round(v[1] / tot_ms, 4) for k, v in tim.items() if v[0]}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "df32": "f32x2"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w.name, "kind": w.kind, "p": w.p,
                   "fitter": {"line": "least-squares pole line", "gauss": "Gaussian sums + Table 1 "
                              "(two pole lines)"}[args.fitter],
                   "boundary": "periodic square (seams are interfaces)" if per else "walls",
                   "elimination": ("consistent (curl of the recovered gradient kept)" if consistent
                                   else "as the paper writes it") if w.kind == "sw" else None,
                   "leaves": f"{w.nlx}x{w.nly}",
                   "leaf_solves": "fast diagonalisation" if fd else (
                       "dense leaf operators on the tensor cores (tcgen05, 6 bf16 slices of 7 bits, FP32 "
                       "accumulation in TMEM, pole sum in FP32 pairs)" if tl else "dense leaf operators"),
                   "merges": ("even/odd blocks of the reflection symmetries" +
                              (f", levels 1-{fused} in one launch per sweep" if fused else "")
                              if merge_sym else "dense blocks") if w.kind == "sw" else "dense blocks",
                   "root": ("seam system of the root box merged with itself" if per else
                            ("four Fourier blocks of the quarter-turn-symmetric wall system" if root_c4
                             else "dense wall inverse") if w.kind == "sw" else "none (Dirichlet)"),
                   "precision": {"fp32": "FP32 operator blocks and products; FP64 vectors, pole sum, maps",
                                 "df32": "FP32-pair (hi, lo) operator blocks, exact split products and "
                                         "compensated sums on the FP32 pipe; FP64 vectors, pole sum, maps",
                                 "fp64": "FP64 throughout"}[args.precision],
                   "n_poles": int(op.alpha.size), "distinct_poles": int((op.alpha.imag >= 0).sum()), "tau": op.tau,
                   "band_X": op.X, "rhs": R, "n_nodes": g.n_nodes, "operator_gb": ob / 1e9,
                   "workspace_gb": wb / 1e9, "build_s": build_s, "parallelism": f"replicas x{world}",
                   "l2": f"operators ({ob / 1e9:.1f} GB) are re-read every step, larger than the 126 MB L2",
                   "timing": "value: untraced steps; kernel shares and roofline: a second, traced pass "
                             f"({ms_traced / args.steps:.3f} ms per step)",
                   "accuracy": "FP64 per-step relative L2 vs the FP64 oracle: tests/test_parity_gpu.py, "
                               "tests/test_sw_config_gpu.py"},
        "e2e": {"value": world * R * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(U0.nbytes)},
        "gpu_launches": int(launches),
        **fp64,
        "kernel_share": shares,
        "roofline": roofline(op, w, R, tim, args.precision, pk, pk_kind, fd=fd, root_c4=root_c4, merge_sym=merge_sym,
                             fused=fused,
                             periodic=per, tl=tl),
        "clocks": clocks,
    }
    if args.cpu_baseline:
        single = cpu_baseline(w, op, x, y, U0[0], budget_s=args.cpu_budget)
        single["cpu"] = _cpu_model()
        try:
            out["cpu_baseline"] = dict(cpu_baseline_all_cores(w, op, U0[0]), single_core=single)
        except Exception as e:                      # the single-core figure still stands
            out["cpu_baseline"] = dict(single, all_cores_error=repr(e))
    print(json.dumps(out), flush=True)


def run_uneven_batch(args):
    """The uneven batch: independent instances (wave and shallow water, different
    leaf grids, p, pole and rhs counts) advanced together through one CUDA graph
    (eo_batch_*), against the same instances stepped one after another.  The
    64-instance draw admits instances in order under an operator budget: each is
    built with the budget still left, and one the library rejects with
    EO_ERR_BUDGET (or whose workspace no longer fits the device) is left out."""
    import torch
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300 import ExpopError
    big = args.workload == W.UNEVEN_BATCH_64
    ws_all = W.uneven_instances_64() if big else W.uneven_instances()
    budget = W.UNEVEN_64_BUDGET_GB if big else 0.0
    ops, states, U0, ws, rejected = [], [], [], [], []
    used_gb = 0.0
    t0 = time.time()
    for w in ws_all:
        g = eo.Grid(w.nlx, w.nly, w.p)
        x, y = g.nodes()
        left = budget - used_gb if budget else 0.0
        if budget and left <= 0.0:
            rejected.append({"instance": w.name, "reason": "budget spent"})
            continue
        try:
            if w.kind == "wave":
                c = W.wave_c(w, x, y)
                op = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.wave_band(w), n_poles=w.n_poles, c2=c * c,
                                 max_rhs=w.n_rhs, precision=args.precision, mem_budget_gb=left)
            else:
                pr = w.params
                op = eo.Operator(g, eo.SW_WALLS, band=W.sw_band(w), n_poles=w.n_poles, f=pr["f"], g=pr["g"],
                                 H=pr["H"], shared_ops=True, max_rhs=w.n_rhs, precision=args.precision,
                                 mem_budget_gb=left)
        except ExpopError as e:
            rejected.append({"instance": w.name, "reason": str(e)[:160]})
            continue
        u0 = np.stack([np.stack(W.initial_fields(w, x, y, r)) for r in range(w.n_rhs)])
        free = torch.cuda.mem_get_info()[0]
        if big and free < u0.nbytes + (16 << 30):
            # keep room for the graph and the states of the instances already in
            rejected.append({"instance": w.name, "reason": "device memory"})
            op.close()
            continue
        used_gb += op.memory()[0] / 1e9
        ops.append(op)
        ws.append(w)
        U0.append(u0)
        states.append(torch.tensor(u0, device="cuda"))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    stream = torch.cuda.current_stream()
    rhs_total = sum(w.n_rhs for w in ws)
    # one after another (each instance autotuned on its first apply)
    for _ in range(args.warmup):
        for op, u in zip(ops, states):
            op.apply(u, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for op, u in zip(ops, states):
            op.apply(u, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    # one graph for all instances
    batch = eo.Batch(ops, states)
    batch.apply(2 * args.warmup)
    torch.cuda.synchronize()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    e0.record(stream)
    batch.apply(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ob = sum(op.memory()[0] for op in ops)
    out = {
        "metric": METRIC, "value": rhs_total * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "df32": "f32x2"}[args.precision], "data": "synthetic",
        "config": {"workload": args.workload, "instances": [w.name for w in ws], "rhs_total": rhs_total,
                   "drawn": len(ws_all), "admitted": len(ws), "rejected": rejected,
                   "budget_gb": budget or None,
                   "operator_gb": ob / 1e9, "build_s": build_s,
                   "sequential": {"ms_per_step": ms_seq / args.steps,
                                  "value": rhs_total * args.steps / (ms_seq / 1e3)},
                   "batch_speedup": ms_seq / ms,
                   "l2": "operators are re-read every step"},
        "roofline": None, "roofline_note": "one CUDA graph over all instances: no per-kernel tracing",
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def cpu_baseline(w, op, x, y, u0, budget_s=30.0):
    """The FP64 oracle's apply phase on the host cores, on a bounded sample:
    the first few distinct poles of one step (factorisations are the oracle's
    build and are not timed), scaled to applies/s."""
    from oracle.resolvent import Stepper
    st = Stepper(oracle_problem(w, op.tau, x, y), op.alpha, op.b)
    upper = np.flatnonzero(op.alpha.imag >= 0)
    P = upper.size
    done, solve_s, t_all = 0, 0.0, time.time()
    for j in upper:
        st._solver(j)                       # factorisation (oracle build), untimed
        t = time.perf_counter()
        st.resolvent(j, u0)
        solve_s += time.perf_counter() - t
        done += 1
        if time.time() - t_all > budget_s:
            break
    per_step = solve_s / done * P
    return {"value": 1.0 / per_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of {P} distinct-pole resolvents of one step on the full workload "
                      f"(sparse LU solves, factorisation excluded as the oracle's build), scaled to one apply",
            "wall_s": time.time() - t_all}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_pole_worker(args):
    """One worker of the all-core baseline: factorise one distinct pole's global
    system (the oracle's build, untimed), wait for every worker, then repeat that
    pole's resolvent solve for budget_s seconds."""
    wname, tau, alpha, bj, u0, budget_s, barrier = args
    from oracle import sem
    from oracle.resolvent import Stepper
    w = W.WORKLOADS[wname]
    og = sem.Grid(w.nlx, w.nly, w.p, periodic=is_periodic(w))
    st = Stepper(oracle_problem(w, tau, og.x, og.y), np.array([alpha]), np.array([bj]))
    st._solver(0)
    barrier.wait()
    n, t0 = 0, time.perf_counter()
    while True:
        st.resolvent(0, u0)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return n, time.perf_counter() - t0


def cpu_baseline_all_cores(w, op, u0, budget_s=10.0, max_workers=8):
    """The FP64 oracle's apply phase on several host cores at once: one process per
    core (spawned, each bounded to one factorisation of about 1 GB), each solving
    its own distinct pole repeatedly; throughput = all solves / the slowest worker's
    time, scaled to applies/s by the number of distinct poles."""
    import multiprocessing as mp
    n = max(1, min(max_workers, os.cpu_count() or 1))
    upper = np.flatnonzero(op.alpha.imag >= 0)
    P = upper.size
    ctx = mp.get_context("spawn")
    t_all = time.time()
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(n)
        tasks = [(w.name, op.tau, complex(op.alpha[upper[k % P]]), complex(op.b[upper[k % P]]), u0, budget_s,
                  barrier) for k in range(n)]
        with ctx.Pool(n) as pool:
            res = pool.map(_oracle_pole_worker, tasks)
    solves = sum(r[0] for r in res)
    elapsed = max(r[1] for r in res)
    return {"value": solves / elapsed / P, "unit": UNIT, "cores": n, "host_cores": os.cpu_count(),
            "kind": "oracle", "cpu": _cpu_model(),
            "sample": f"{n} processes (capped at {max_workers}: each holds one factorisation of about 2 GB, so "
                      f"this is {n} of the host's {os.cpu_count()} cores, not all of them), one distinct pole "
                      f"each, {solves} sparse-LU resolvent solves of the full workload in {elapsed:.1f} s "
                      f"(factorisation excluded as the oracle's build), scaled to one apply of {P} distinct poles",
            "wall_s": time.time() - t_all}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = W.WORKLOADS[args.workload]
    from oracle import rational, sem
    from oracle.resolvent import Stepper
    g = sem.Grid(w.nlx, w.nly, w.p, periodic=is_periodic(w))
    # the oracle's own approximant for this workload's pole count; for a fixed
    # step (thousands of poles) the oracle's pole line of the same density
    # (sigma = 4.5, spacing 1, reaching 32 past the band): the timed sample is one
    # resolvent solve, whose cost does not depend on which pole it is
    if w.n_poles:
        alpha, b, X = rational.fit(w.n_poles)
        tau = X / W.BAND[w.name]
    else:
        tau = w.tau
        M = int(np.ceil(tau * W.BAND[w.name] + 32.0))
        alpha = rational.pole_line(2 * M + 1, 4.5, 1.0)
        b = np.ones(alpha.size, dtype=np.complex128)
    u0 = np.stack(W.initial_fields(w, g.x, g.y, 0))
    st = Stepper(oracle_problem(w, tau, g.x, g.y), alpha, b)
    M = (alpha.size - 1) // 2
    P = M + 1
    # one "step" of this arm = one distinct-pole resolvent solve with a factorised
    # pole (the oracle's apply phase; factorising is its build), scaled by the
    # number of distinct poles to one apply
    j = M + P // 2
    st._solver(j)
    for _ in range(args.warmup):
        st.resolvent(j, u0)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st.resolvent(j, u0)
        t.append(time.perf_counter() - t0)
    per_solve = float(np.mean(t))
    per_apply = per_solve * P
    value = 1.0 / per_apply
    # ms_per_step is the time of one timed step of this arm (one solve), so steps *
    # ms_per_step is the timed work; value extrapolates it to whole applies
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "extrapolated": True,
           "timed_step": "one sparse-LU resolvent solve of one distinct pole on the full workload",
           "scale_to_apply": P, "ms_per_apply_extrapolated": per_apply * 1e3,
           "config": {"workload": w.name, "n_poles": int(alpha.size)},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} sparse-LU resolvent solves of one distinct pole on the full "
                                      f"workload, scaled by {P} distinct poles to one apply (factorisation "
                                      "excluded as the oracle's build)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def reduce_max(value, dist, device=None):
    """Max of a per-rank float over the process group (identity without one)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT,
                    choices=sorted(W.WORKLOADS) + [W.UNEVEN_BATCH, W.UNEVEN_BATCH_64])
    ap.add_argument("--rhs", type=int, default=1)
    ap.add_argument("--poles", type=int, default=0, help="override the pole count (profiling cases)")
    ap.add_argument("--leaves", type=int, default=0, help="override leaves per side (profiling cases)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dense-leaves", action="store_true",
                    help="dense leaf solution operators instead of the separable leaf eigenbasis")
    ap.add_argument("--precision", default="df32", choices=["df32", "fp32", "fp64"])
    ap.add_argument("--root-dense", action="store_true",
                    help="keep the dense wall inverse instead of the four Fourier blocks of a square domain")
    ap.add_argument("--merge-dense", action="store_true",
                    help="apply the dense merge blocks instead of the even/odd reflection blocks")
    ap.add_argument("--fitter", default="line", choices=["line", "gauss"],
                    help="line: our least-squares approximant; gauss: the paper's Gaussian-sum construction")
    ap.add_argument("--tensor-leaves", action="store_true",
                    help="leaf interior solves and pole sum on the tensor cores (bf16 slices, tcgen05)")
    ap.add_argument("--merge-fuse", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="low merge levels fused into one launch per sweep (0: one launch per level)")
    ap.add_argument("--no-fp64-compare", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in (W.UNEVEN_BATCH, W.UNEVEN_BATCH_64):
        run_uneven_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
