#!/usr/bin/env python
"""Benchmark of the Modal Gamma' projection on one or more GB300s.

One step = one full separable projection (Gauss-Legendre nodes, weighted
Legendre table, l contraction, triple product with the slice reduction,
symmetrise/gather) of the Planck-scale workload: l_max = 2000, 20 basis
functions (1540 modes each side), 500 radial points, N_mu = 3001, i.e.
1,500,500 (x, mu) slices.  The metric is slices per second of the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Under torchrun (N > 1) every rank projects its own independent problem (a
different seed): weak scaling with no collective on the data path; the time
is the max over ranks.  With --shard x the ranks split the radial points of
ONE problem and sum Gamma' with an all-reduce (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Γ_nm (x,μ)-slices/s and % tensor peak vs plain FP64 GPU at stated error"
PREC = {"fp64": 0, "fp32": 1, "ozaki": 2, "tf32": 3, "bf16x3": 4}
DTYPE = {"fp64": "f64", "fp32": "f32", "ozaki": "bf16x(ozaki)+f64", "tf32": "tf32+f32", "bf16x3": "bf16x3+f32"}
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates of the part
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (CUDA cores), nominal figure
FP32_TFLOPS = 73.3           # GB300 FP32 FMA rate measured on this machine with an FMA-chain kernel
TC_SLICE_PRODUCTS = 15       # BF16 slice products per useful MAC in the tensor-core form
# DRAM bytes (read + write) per launch of the workload's size, from one ncu
# capture (n_x = 8 gives one launch with the same K as every launch of the
# 500-point step), keyed by the kernel's form.  A form that changed since its
# capture is left out (its traffic is then reported as null).
NCU_TRAFFIC = {("tc_gemm_triple", "single"): 7.136e9 + 92.5e6, ("tc_make_Y", "single"): 80.6e6 + 5.497e9,
               ("tc_make_Y", "pair"): 80.6e6 + 5.497e9, ("tc_make_Y", "queue"): 80.6e6 + 5.497e9,
               ("tc_gemm_triple", "tail"): 3.112e9 + 15.7e6}  # tail form: per half-chunk launch
# Tensor-pipe activity of the triple GEMM from one full ncu capture of a
# half-chunk launch of the tail form (255 whole tiles, K = 12004): cycles with
# the pipe busy over the SMs' active cycles and over the elapsed cycles.  It
# does not depend on the SM clock, unlike `frac` against the measured cuBLAS
# peak, whose clock under load differs from this kernel's.  Like
# NCU_TRAFFIC, valid only while the kernel is unchanged since the capture.
NCU_TENSOR = {("tc_gemm_triple", "tail"): {"of_active_cycles": 0.680, "of_elapsed_cycles": 0.554}}
# kernels inside one profiler scope (the library counts kernels; a roofline
# divides the scope's time by its scope count)
SCOPE_KERNELS = {"tc_make_Y": 2, "tc_prep_M": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", *PREC],
                    help="auto: the tensor-core form (ozaki) for every workload (the gradient "
                         "workload's adjoint included)")
    ap.add_argument("--n-x", type=int, default=500, help="radial points (workload: 500)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="planck",
                    choices=["planck", "grad", "batched", "direct", "full", "integrators", "sparse"],
                    help="planck: the headline line; grad: forward + adjoint at l_max 1000 / "
                         "16 functions / 300 x; batched: 64 uneven models in one call; direct: "
                         "the Planck problem by the tetrahedral sum on the sparse l grid; full: "
                         "Gamma' + the Gram matrix + the Cholesky solve (the full Gamma); "
                         "integrators: accuracy against time of the two radial rules; sparse: "
                         "dense-against-sparse error curves of the direct form")
    ap.add_argument("--tc-fused", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core triple product: 0 = Y through HBM, 1 and 2 = Y formed in "
                         "shared memory (two forms)")
    ap.add_argument("--shard", default="none", choices=["none", "x"],
                    help="none: one independent problem per rank (weak scaling); x: the radial "
                         "points of one problem split over the ranks, Gamma' summed by an "
                         "all-reduce (strong scaling)")
    ap.add_argument("--x-chunk", type=int, default=0,
                    help="radial points per streamed chunk (0: the library's choice)")
    ap.add_argument("--tc-queue", type=int, default=0, choices=[0, 1],
                    help="tensor-core triple product GEMM as a persistent kernel over a work queue: 1")
    ap.add_argument("--tc-overlap", type=int, default=0,
                    help="SMs left to the Y pass running beside the queue GEMM (0: no overlap)")
    ap.add_argument("--tc-tail", type=int, default=1, choices=[0, 1],
                    help="operand and Y passes beside the previous chunk's GEMM on a second stream: 1 (default)")
    ap.add_argument("--tc-split-k", type=int, default=0,
                    help="K splits of the tensor-core triple GEMM (0: the library's choice)")
    ap.add_argument("--tc-pair", type=int, default=0, choices=[0, 1],
                    help="tensor-core triple product GEMM on CTA pairs (2-SM MMA): 1, or single CTAs: 0")
    ap.add_argument("--direct-tensor", type=int, default=0, choices=[0, 1, 2],
                    help="direct workload on the tensor cores (BF16 slices): 1 the Gamma' update, "
                         "2 also the radial integrals; 0: FP64")
    ap.add_argument("--once", action="store_true",
                    help="run one projection and exit (a small case for profiler captures)")
    ap.add_argument("--fp64-x", type=int, default=20,
                    help="radial points of the plain-FP64 comparison run (0: skip; for the direct "
                         "workload, 0 skips its FP64 comparison call)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_setup(backend_gpu: bool):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if backend_gpu else "gloo")
    return ws, rank, local


def max_over_ranks(v: float, ws: int, device=None) -> float:
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
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
        self.f.flush()
        rows = []
        for line in Path(self.f.name).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        load = [r for r in rows if r[0] > 0.5 * r[1]] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return json.loads(p.read_text()), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
def cpu_baseline(P, seconds: float):
    """The FP64 oracle as it stands, on a bounded sample of the workload: the
    radial points nearest the last-scattering peak and the first K
    Gauss-Legendre nodes, all 1540 x 1540 modes, sized for ~`seconds` of work.
    Returns (slices/s, seconds, sample description, threads)."""
    import oracle
    import synthetic as syn
    mu, om = oracle.gl_nodes(P.n_mu)
    order = np.argsort(np.abs(P.x - syn.X_PEAK))

    def run(nx, k):
        idx = np.sort(order[:nx])
        Ps = syn.Problem(**{**P.__dict__, "qt": P.qt[idx].copy(), "x": P.x[idx], "n_x": nx})
        t0 = time.perf_counter()
        oracle.separable(Ps, xw=np.ones(nx), mu=mu[:k], om=om[:k])
        return time.perf_counter() - t0

    k0 = min(64, P.n_mu)
    per_slice = run(1, k0) / k0
    want = max(1, int(seconds / max(per_slice, 1e-9)))
    nx = min(P.n_x, max(1, want // P.n_mu))
    k = P.n_mu if want >= P.n_mu else want
    t = run(nx, k)
    desc = (f"{nx} of {P.n_x} radial points x first {k} of {P.n_mu} GL nodes, all "
            f"{P.n_late}x{P.n_prim} modes ({t:.1f} s)")
    return nx * k / t, t, desc, oracle.num_threads()


def run_reference(args):
    ws, rank, _ = dist_setup(False)
    if rank != 0:
        return
    import synthetic as syn
    P = syn.planck_size(n_x=args.n_x)
    vals = []
    desc, cores = "", 1
    for i in range(args.warmup + args.steps):
        v, t, desc, cores = cpu_baseline(P, args.cpu_seconds / max(1, args.steps))
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    sample = desc + " per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "slices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * P.slices / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": P.name, "l_max": P.l_max, "nb": P.nb_late, "n_x": P.n_x,
                       "n_mu": P.n_mu, "slices": P.slices},
            "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1503_08809_gb300 as mg
    import synthetic as syn

    prec_name = "ozaki" if args.precision == "auto" else args.precision
    prec = PREC[prec_name]
    sharded = args.shard == "x"
    P = syn.planck_size(seed=1 if sharded else 1 + rank, n_x=args.n_x)
    h = mg.Handle(dev)
    mg.set_option(mg.OPT_TC_TRIPLE_FUSED, args.tc_fused, handle=h)
    mg.set_option(mg.OPT_TC_PAIR, args.tc_pair, handle=h)
    mg.set_option(mg.OPT_TC_QUEUE, args.tc_queue, handle=h)
    mg.set_option(mg.OPT_TC_OVERLAP, args.tc_overlap, handle=h)
    mg.set_option(mg.OPT_TC_SPLIT_K, args.tc_split_k, handle=h)
    mg.set_option(mg.OPT_TC_OVERLAP_TAIL, args.tc_tail, handle=h)
    dp = mg.DeviceProblem.from_host(P, device=dev, handle=h)
    gamma = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)

    def step():
        if sharded:
            mg.project_separable_sharded(dp, rank, ws, precision=prec, out=gamma, handle=h)
        else:
            mg.project_separable(dp, precision=prec, out=gamma, handle=h, x_chunk=args.x_chunk)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # ---- device-timed region (profiler events on, clocks sampled) ----------
    lib = mg.lib()
    lib.modal_profile_enable(h.ptr, 1)
    import ctypes
    names = ctypes.create_string_buffer(32 * 64)
    launches = (ctypes.c_int64 * 64)()
    tms = (ctypes.c_double * 64)()
    nout = ctypes.c_int32()
    lib.modal_profile_read(h.ptr, 64, names, launches, tms, ctypes.byref(nout))  # reset
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    lib.modal_profile_read(h.ptr, 64, names, launches, tms, ctypes.byref(nout))
    lib.modal_profile_enable(h.ptr, 0)
    prof = {}
    for i in range(nout.value):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
        prof[nm] = (int(launches[i]), float(tms[i]))
    ms_max = max_over_ranks(ms, ws, dev)
    job_slices = P.slices if sharded else ws * P.slices
    value = job_slices / (ms_max * 1e-3)

    # ---- rooflines: the dominant kernel, and every tensor / HBM kernel ------
    peaks, src = measured_peaks()
    launches_per_step = {k: max(1, v[0] // args.steps) for k, v in prof.items()}
    form = ("pair" if args.tc_pair else "queue" if (args.tc_queue or args.tc_overlap) else
            "tail" if (args.tc_tail and prec_name == "ozaki" and not sharded) else "single")
    rooflines = {k: kernel_roofline(k, prof[k], launches_per_step[k], P, prec_name, peaks, src, args.steps, ms,
                                    form) for k in prof}
    rooflines = {k: v for k, v in rooflines.items() if v is not None}
    dom = max(prof, key=lambda k: prof[k][1]) if prof else None
    roof = rooflines.get(dom)
    gpu_launches = sum(v[0] for v in prof.values())
    step_tensor = None
    if prec_name == "ozaki":
        # the whole step's issued tensor work (triple product and l contraction)
        # over the step time: the path's own fraction of the tensor peak
        g2 = P.nb_prim * (P.nb_prim + 1) // 2
        macs = g2 * P.nb_prim * P.n_late + P.nb_late * P.nb_prim * P.L
        tf = TC_SLICE_PRODUCTS * 2.0 * macs * P.slices / (ms * 1e-3) / 1e12
        step_tensor = {"issued_tflops": tf, "peak": peaks["bf16_tflops"], "frac": tf / peaks["bf16_tflops"],
                       "peak_source": f"bf16 {src}"}
    if form == "tail" and roof is not None and dom == "tc_gemm_triple":
        # under the tail overlap the GEMM's launches share the SMs with the next
        # chunk's operand passes, so its launch time is not the kernel's own:
        # two more steps with one stream give that figure
        mg.set_option(mg.OPT_TC_OVERLAP_TAIL, 0, handle=h)
        p2 = profiled(h, lambda: [step() for _ in range(2)], dev)
        mg.set_option(mg.OPT_TC_OVERLAP_TAIL, 1, handle=h)
        if "tc_gemm_triple" in p2:
            alone = kernel_roofline("tc_gemm_triple", p2["tc_gemm_triple"],
                                    max(1, p2["tc_gemm_triple"][0] // 2), P, prec_name, peaks, src, 2, ms,
                                    "single")
            roof["alone"] = {k: alone[k] for k in ("achieved", "frac", "kernel_ms_avg", "traffic")}
            roof["note"] = ("launch time includes the next chunk's operand and Y passes sharing the SMs "
                            "(MODAL_OPT_TC_OVERLAP_TAIL); 'alone': the same kernel with one stream")

    # ---- end to end through host buffers -----------------------------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hq, hqt, hw, hx = pin(P.q), pin(P.qt), pin(P.w_l), pin(P.x)
        hl, hp = pin(P.late_modes), pin(P.prim_modes)
        hg = torch.empty(P.n_late, P.n_prim, dtype=torch.float64).pin_memory()
        dq, dqt, dw, dx = (torch.empty_like(t, device=dev) for t in (hq, hqt, hw, hx))
        dl, dpm = torch.empty_like(hl, device=dev), torch.empty_like(hp, device=dev)
        h2d = sum(t.numel() * t.element_size() for t in (hq, hqt, hw, hx, hl, hp))
        d2h = hg.numel() * hg.element_size()

        def e2e_step():
            for d, s in ((dq, hq), (dqt, hqt), (dw, hw), (dx, hx), (dl, hl), (dpm, hp)):
                d.copy_(s, non_blocking=True)
            xw = mg.x_weights(dx, handle=h)
            dpe = mg.DeviceProblem(dq, dqt, dw, xw, dl, dpm, P.l_min, P.l_max, dev)
            if sharded:
                g = mg.project_separable_sharded(dpe, rank, ws, precision=prec, out=gamma, handle=h)
            else:
                g = mg.project_separable(dpe, precision=prec, out=gamma, handle=h)
            hg.copy_(g, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        barrier(ws)
        e0.record(st)
        for _ in range(args.steps):
            e2e_step()
        e1.record(st)
        torch.cuda.synchronize(dev)
        barrier(ws)
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws, dev)
        e2e = {"value": job_slices / (ms_e2e * 1e-3), "unit": "slices/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        return
    # ---- plain FP64 GPU path and the stated error -------------------------
    fp64 = err = None
    if args.fp64_x > 0 and prec_name != "fp64":
        fp64, err = fp64_comparison(P, args.fp64_x, prec, value, dev, h)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, t, desc, cores = cpu_baseline(P, args.cpu_seconds)
        cpu = {"value": v, "unit": "slices/s", "cores": cores, "kind": "oracle", "sample": desc}
    line = {"metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": DTYPE[prec_name], "data": "synthetic",
            "config": {"workload": P.name, "l_max": P.l_max, "nb": P.nb_late, "n_x": P.n_x,
                       "n_mu": P.n_mu, "slices": P.slices, "precision": prec_name,
                       "n_modes": P.n_late, "tc_triple": ["Y through HBM", "shared-memory Y",
                                                          "shared-memory Y (16 warps)"][args.tc_fused],
                       "tc_gemm": ("CTA pairs (2-SM MMA)" if args.tc_pair else
                                   f"persistent work queue on {152 - args.tc_overlap} SMs, Y pass beside it"
                                   if args.tc_overlap else
                                   "persistent work queue" if args.tc_queue else
                                   "one CTA per tile (or per K range of a tile)" + (f", {args.tc_split_k} K splits"
                                                                                     if args.tc_split_k else "") +
                                   (", operand and Y passes beside the previous chunk's GEMM" if args.tc_tail
                                    else "")),
                       "g_layout": "blocks by the middle index, each expanded along its wider side",
                       "l2": "inputs larger than L2 (q~ 160 MB; M chunks of up to 2 GiB)",
                       "parallelism": (f"x-sharded over {ws} ranks, FP64 all-reduce of Gamma'" if sharded
                                       else f"{ws} independent problem(s)")},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "fp64_gpu": fp64, "error": err, "kernel_rooflines": rooflines, "step_tensor": step_tensor,
            "clocks": clk, "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}}
    print(json.dumps(line), flush=True)


def kernel_roofline(name, rec, per_step, P, prec_name, peaks, src, steps, ms, form="single"):
    """Achieved algorithmic work per launch / mean launch time against the
    measured peak of the unit that bounds the kernel (None if not modelled)."""
    nl, tot = rec
    nl = max(1, nl // SCOPE_KERNELS.get(name, 1))
    per_step = max(1, per_step // SCOPE_KERNELS.get(name, 1))
    avg_s = tot / nl * 1e-3
    g2 = P.nb_prim * (P.nb_prim + 1) // 2
    gsize = g2 * P.nb_prim * P.n_late          # useful MACs per slice of the triple product
    k = P.slices / per_step                     # slices per launch
    kpad = math.ceil(k / 64) * 64
    extra = {}
    if name.startswith("triple_") or name.startswith("contract_l_"):
        macs = gsize if name.startswith("triple_") else P.nb_late * P.nb_prim * P.L
        work, unit, bound = 2.0 * macs * k, "TFLOP/s", "alu"
        peak, note = (FP64_NOMINAL_TFLOPS, "fp64 nominal") if name.endswith("f64") else \
            (FP32_TFLOPS, "fp32 measured (FMA chain)")
    elif name in ("tc_gemm_triple", "tc_gemm_l"):
        macs = gsize if name == "tc_gemm_triple" else P.nb_late * P.nb_prim * P.L
        work, unit, bound = TC_SLICE_PRODUCTS * 2.0 * macs * k, "TFLOP/s", "tensor"
        peak, note = peaks["bf16_tflops"], f"bf16 {src}"
        extra = {"flops_counted": f"issued tensor flops ({TC_SLICE_PRODUCTS} BF16 slice products "
                                  "per useful MAC)",
                 "useful_achieved": 2.0 * macs * k / avg_s / 1e12}
    elif name in ("fa_gemm_l_tf32", "fa_gemm_l_bf16x3"):
        # the l contraction with FP32 accumulation: 1 TF32 or 3 BF16 products per useful MAC
        macs = P.nb_late * P.nb_prim * P.L
        nprod = 1 if name.endswith("tf32") else 3
        k_launch = P.slices / per_step           # slices per launch
        work, unit, bound = nprod * 2.0 * macs * k_launch, "TFLOP/s", "tensor"
        if name.endswith("tf32"):
            peak, note = peaks["bf16_tflops"] * NOMINAL_TF32_OVER_BF16, f"tf32 = bf16 {src} x nominal 1.1/2.25"
        else:
            peak, note = peaks["bf16_tflops"], f"bf16 {src}"
        extra = {"flops_counted": f"issued tensor flops ({nprod} product(s) per useful MAC)",
                 "useful_achieved": 2.0 * macs * k_launch / avg_s / 1e12}
    elif name == "tc_make_Y":
        # Y rows of the pairs the G layout of the Y-in-HBM forms uses: (a, b)
        # for b < h and (b, c) for b >= h, h = ceil(nb / 2)
        hh = (P.nb_late + 1) // 2
        rows = g2 * (hh * (hh + 1) // 2 + (P.nb_late - hh) * (P.nb_late - hh + 1) // 2)
        work = 10.0 * rows * kpad + 8.0 * P.nb_late * P.nb_prim * kpad   # Y slices out, M~ in
        unit, bound, peak, note = "GB/s", "hbm", peaks["hbm_gbs"], f"hbm copy {src}"
    else:
        return None
    scale = 1e9 if bound == "hbm" else 1e12
    achieved = work / avg_s / scale
    r = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
         "frac": achieved / peak, "traffic": NCU_TRAFFIC.get((name, form)) if P.n_x == 500 else None,
         "peak_source": note, "kernel_ms_avg": avg_s * 1e3, "launches_per_step": per_step,
         "kernel_share_of_step": tot / (ms * steps)}
    if (name, form) in NCU_TENSOR:
        r["ncu_tensor_active"] = NCU_TENSOR[(name, form)]
    r.update(extra)
    return r


def entry_errors(g, ref):
    """Normwise max|dG| / max|G_ref|, and entrywise relative errors with a
    floor of 1e-12 max|G_ref| (max and RMS).  The caller adds the conditioned
    check, max |dG| / (the same sum taken in magnitude)."""
    d = np.abs(g - ref)
    scale = np.abs(ref).max()
    rel = d / np.maximum(np.abs(ref), 1e-12 * scale)
    return {"normwise": float(d.max() / scale), "max_rel": float(rel.max()),
            "rms_rel": float(np.sqrt(np.mean(rel ** 2)))}


def fp64_comparison(P, n_x, prec, value, dev, h):
    """The plain FP64 GPU path on the `n_x` radial points of the workload
    nearest the last-scattering peak (its time is linear in the slice count),
    timed once after a warm-up, and the error of the timed precision against
    it on those inputs."""
    import torch
    import paper_1503_08809_gb300 as mg
    import synthetic as syn
    idx = np.sort(np.argsort(np.abs(P.x - syn.X_PEAK))[:n_x])  # the radial points nearest the peak
    Ps = syn.Problem(**{**P.__dict__, "qt": P.qt[idx].copy(), "x": P.x[idx], "n_x": n_x})
    dp = mg.DeviceProblem.from_host(Ps, device=dev, handle=h)
    st = torch.cuda.current_stream(dev)
    ref = mg.project_separable(dp, precision=PREC["fp64"], handle=h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    ref = mg.project_separable(dp, precision=PREC["fp64"], handle=h)
    e1.record(st)
    torch.cuda.synchronize(dev)
    v64 = Ps.slices / (e0.elapsed_time(e1) * 1e-3)
    scale = torch.empty_like(ref)          # per-entry error scale (untimed)
    mg.project_separable(dp, precision=PREC["fp64"], handle=h, error_estimate=scale)
    g = mg.project_separable(dp, precision=prec, handle=h)
    mg.handle_status(handle=h)
    fp64 = {"value": v64, "unit": "slices/s", "sample": f"{n_x} of {P.n_x} radial points (nearest the peak), "
            f"all {P.n_mu} GL nodes and {P.n_late}x{P.n_prim} modes", "speedup": value / v64}
    gn, rn, sn = g.cpu().numpy(), ref.cpu().numpy(), scale.cpu().numpy()
    err = {"vs": "plain FP64 GPU path (itself within 1e-10 of the oracle) on the same sample",
           **entry_errors(gn, rn),
           "conditioned_max": float((np.abs(gn - rn) / np.maximum(sn, 1e-300)).max())}
    return fp64, err


def run_once(args):
    """One projection of the workload (with --n-x radial points), no timing."""
    import torch
    import paper_1503_08809_gb300 as mg
    import synthetic as syn
    prec = PREC["ozaki" if args.precision == "auto" else args.precision]
    P = syn.planck_size(n_x=args.n_x)
    mg.set_option(mg.OPT_TC_TRIPLE_FUSED, args.tc_fused)
    mg.set_option(mg.OPT_TC_PAIR, args.tc_pair)
    mg.set_option(mg.OPT_TC_QUEUE, args.tc_queue)
    mg.set_option(mg.OPT_TC_OVERLAP, args.tc_overlap)
    g = mg.project_separable(mg.DeviceProblem.from_host(P), precision=prec)
    if prec == PREC["ozaki"]:
        mg.handle_status()
    torch.cuda.synchronize()
    print(json.dumps({"once": P.name, "max_abs_gamma": float(g.abs().max())}))


def sparse_triples(lg, parity: bool = True) -> int:
    """Sorted triples l1 <= l2 <= l3 of the grid with the triangle condition
    and (with ``parity``) even l1 + l2 + l3: the nonzero terms of the
    exact-3j direct sum, or of the Gosper form without parity."""
    lg = np.asarray(lg, dtype=np.int64)
    n = 0
    for i in range(lg.size):
        l1 = lg[i]
        l2 = lg[i:, None]
        l3 = lg[None, i:]
        ok = (l3 >= l2) & (l3 <= l1 + l2)
        if parity:
            ok &= (l1 + l2 + l3) % 2 == 0
        n += int(np.count_nonzero(ok))
    return n


SPARSE_STEPS = (20, 10, 5, 3)


def run_sparse(args):
    """Dense-against-sparse error curves of the direct form (Eq. 3D) on
    multipole grids: every l to 50 then every s-th l (s = 20, 10, 5, 3) at
    l_max 1000 / 16 functions / 100 x against the dense Gamma' (separable
    form, FP64), and the 334-point grid at Planck size against the dense
    Gamma' (tensor-core form, error ~1e-9), each with exact 3j^2 weights
    (triangle + parity, weight prod dw) and the Gosper form (1/2 Gosper,
    triangle only).  Error: relative RMS error (%) of the unit-normalised matrix and
    the normwise max|dGamma|/max|Gamma|; time of each direct call."""
    import torch
    import paper_1503_08809_gb300 as mg
    import synthetic as syn
    dev = torch.device("cuda", 0)
    h = mg.Handle(dev)
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(f):
        torch.cuda.synchronize(dev)
        e0, e1 = ev(), ev()
        e0.record(st)
        out = f()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return out.cpu().numpy(), e0.elapsed_time(e1)

    def errs(g, ref):
        u = lambda a: a / np.sqrt((a ** 2).sum())
        return {"rel_rms_pct": 100.0 * float(np.sqrt(((u(g) - u(ref)) ** 2).sum())),
                "normwise": float(np.abs(g - ref).max() / np.abs(ref).max())}

    study, tot_tr, tot_ms = {}, 0, 0.0
    cases = [("lmax1000_nb16_nx100", syn.make_problem(1000, 16, 100), mg.PREC_FP64,
              [(f"step{s}", *syn.stepped_l_grid(1000, s)) for s in SPARSE_STEPS]),
             ("lmax2000_nb20_nx500", syn.planck_size(), mg.PREC_OZAKI_BF16,
              [("planck334", *syn.sparse_l_grid(2000))])]
    for name, P, dprec, grids in cases:
        dp = mg.DeviceProblem.from_host(P, device=dev, handle=h)
        ref, ref_ms = timed(lambda: mg.project_separable(dp, precision=dprec, handle=h))
        if dprec == mg.PREC_OZAKI_BF16:
            mg.handle_status(handle=h)
        rows = {}
        for gname, lg, dw in grids:
            row = {"points": int(lg.size)}
            for mode, mname in ((mg.W_EXACT_3J, "exact"), (mg.W_SMOOTH_GOSPER, "gosper")):
                g, ms = timed(lambda: mg.project_direct(dp, lg, dw, mode, handle=h))
                tr = sparse_triples(lg, parity=mode == mg.W_EXACT_3J)
                row[mname] = {**errs(g, ref), "triples": tr, "ms": ms}
                tot_tr += tr
                tot_ms += ms
            rows[gname] = row
        study[name] = {"dense_reference": ("separable FP64" if dprec == mg.PREC_FP64 else
                                           "separable tensor-core form"), "dense_ms": ref_ms,
                       "grids": rows}
    cfg = {"workload": "direct form on sparse l grids against the dense Gamma'", "study": study,
           "error": "relative RMS error (%) of the unit-normalised Gamma' (100 |G/|G| - R/|R||_F) "
                    "and normwise max|G - R| / max|R|"}
    print(json.dumps({"metric": METRIC, "value": tot_tr / (tot_ms * 1e-3), "unit": "triples/s",
                      "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": tot_ms,
                      "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": cfg}), flush=True)


def run_extra(args):
    """The gradient and batched workloads (one GPU; printed as one JSON line)."""
    import ctypes
    import torch
    import paper_1503_08809_gb300 as mg
    import synthetic as syn
    dev = torch.device("cuda", 0)
    # auto: the tensor-core form (forward and adjoint) for every workload
    prec_name = args.precision if args.precision != "auto" else "ozaki"
    prec = PREC[prec_name]
    h = mg.Handle(dev)
    mg.set_option(mg.OPT_TC_PAIR, args.tc_pair, handle=h)
    mg.set_option(mg.OPT_TC_QUEUE, args.tc_queue, handle=h)
    st = torch.cuda.current_stream(dev)
    unit = "slices/s"
    if args.workload == "grad":
        P = syn.grad_size()
        dp = mg.DeviceProblem.from_host(P, device=dev, handle=h)
        gbar = torch.tensor(syn.random_cotangent(P.n_late, P.n_prim, seed=4), device=dev)
        slices = P.slices
        bprec = prec          # the adjoint in the same form (tensor-core adjoint for ozaki)

        def step():
            mg.project_separable(dp, precision=prec, handle=h)
            mg.project_backward(dp, gbar, precision=bprec, handle=h)
        cfg = {"workload": P.name, "l_max": P.l_max, "nb": P.nb_late, "n_x": P.n_x, "n_mu": P.n_mu,
               "slices": slices, "precision": prec_name, "backward_precision":
               [k for k, v in PREC.items() if v == bprec][0], "step": "forward + adjoint"}
    elif args.workload == "direct":
        P = syn.planck_size()
        dp = mg.DeviceProblem.from_host(P, device=dev, handle=h)
        lg, dw = syn.sparse_l_grid(P.l_max)
        slices = sparse_triples(lg)          # the unit here: (l1 <= l2 <= l3) triples
        unit = "triples/s"

        mg.set_option(mg.OPT_DIRECT_TENSOR, args.direct_tensor, handle=h)
        gdir = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dev)

        def step():
            mg.project_direct(dp, lg, dw, out=gdir, handle=h)
        cfg = {"workload": P.name + "_sparse_direct", "l_max": P.l_max, "nb": P.nb_late, "n_x": P.n_x,
               "grid_points": int(lg.size), "triples": slices, "weight": "exact 3j^2",
               "tensor_cores": ["none", "Gamma' update", "radial integrals and Gamma' update"][args.direct_tensor],
               "step": "one direct projection (Eq. 3D) on the sparse grid"}
    elif args.workload == "full":
        P = syn.planck_size()
        dp = mg.DeviceProblem.from_host(P, device=dev, handle=h)
        wg = torch.tensor(syn.gram_weights(P.l_min, P.l_max), device=dev)
        # With this synthetic basis the Gram matrix is singular to FP64, so its
        # factorisation stops early; the solve is timed on a well-conditioned
        # SPD matrix of the same order instead (same launches and work).
        rng = np.random.default_rng(5)
        B = torch.tensor(rng.standard_normal((P.n_late, P.n_late)), device=dev)
        S = B @ B.T / P.n_late + torch.eye(P.n_late, dtype=torch.float64, device=dev)
        gp = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dev)
        G = torch.empty(P.n_late, P.n_late, dtype=torch.float64, device=dev)
        X = torch.empty_like(gp)
        slices = P.slices + P.n_mu          # Gamma' slices + the Gram matrix's (one radial point)
        parts = {
            "separable": lambda: mg.project_separable(dp, precision=prec, out=gp, handle=h),
            "gram": lambda: mg.gram(dp, wg, precision=prec, out=G, handle=h),
            "solve": lambda: mg.gram_solve(S, gp, out=X, handle=h, raise_if_not_pd=False),
        }

        def step():
            for f in parts.values():
                f()
        cfg = {"workload": P.name + "_full_gamma", "l_max": P.l_max, "nb": P.nb_late, "n_x": P.n_x,
               "n_mu": P.n_mu, "slices": slices, "precision": prec_name,
               "step": "Gamma' + Gram matrix + Cholesky solve (n = m = 1540, FP64)",
               "solve_matrix": "SPD stand-in of the Gram's order: the synthetic basis's Gram "
                               "matrix is singular to FP64"}
    else:
        probs = syn.batched_models(64)
        dps = [mg.DeviceProblem.from_host(P, device=dev, handle=h) for P in probs]
        outs = [torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dev) for P in probs]
        slices = sum(P.slices for P in probs)

        def step():
            mg.project_separable_batched(dps, precision=prec, outs=outs, handle=h)
        cfg = {"workload": "64 models: l_max U[500,2500], 10-20 functions, 200-600 x",
               "slices": slices, "precision": prec_name, "step": "one batched call (CUDA graph)"}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    if prec == PREC["ozaki"]:
        mg.handle_status(handle=h)
    ms = e0.elapsed_time(e1) / args.steps
    if args.workload == "batched":
        cfg["fp64_sequential"] = fp64_sequential(probs, dps, slices / (ms * 1e-3), dev, h)
    if args.workload == "direct":
        prof = profiled(h, step, dev)
        cfg["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}
        if args.direct_tensor and args.fp64_x:  # the same call in FP64 throughout, for the error
            mg.handle_status(handle=h)
            g = gdir.clone()
            mg.set_option(mg.OPT_DIRECT_TENSOR, 0, handle=h)
            mg.project_direct(dp, lg, dw, out=gdir, handle=h)
            cfg["error_vs_fp64"] = float((g - gdir).abs().max() / gdir.abs().max())
    if args.workload == "grad":             # forward alone, and the error of the adjoint vs FP64
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(args.steps):
            mg.project_separable(dp, precision=prec, handle=h)
        e1.record(st)
        torch.cuda.synchronize(dev)
        cfg["forward_ms"] = e0.elapsed_time(e1) / args.steps
        cfg["adjoint_ms"] = ms - cfg["forward_ms"]
        dqt, dq = mg.project_backward(dp, gbar, precision=bprec, handle=h)
        if bprec == PREC["ozaki"]:
            mg.handle_status(handle=h)
        dqt64, dq64 = mg.project_backward(dp, gbar, handle=h)
        nw = lambda a, b: float((a - b).abs().max() / b.abs().max())
        cfg["adjoint_error_vs_fp64"] = {"dqt_normwise": nw(dqt, dqt64), "dq_normwise": nw(dq, dq64)}
        # per-kernel times of one step (the library's CUDA-event profiler) and
        # the adjoint's dL/dM GEMM against the BF16 peak
        prof = profiled(h, step, dev)
        cfg["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}
        if "adj_gemm_dM" in prof and bprec == PREC["ozaki"]:
            nl, tot = prof["adj_gemm_dM"]
            p2l, p2p = P.nb_late * (P.nb_late + 1) // 2, P.nb_prim * (P.nb_prim + 1) // 2
            macs = P.slices * P.nb_late * P.nb_prim * p2l * p2p       # per step: slices x (x,y) x Y rows
            peaks, src = measured_peaks()
            achieved = TC_SLICE_PRODUCTS * 2.0 * macs / (tot * 1e-3) / 1e12
            cfg["roofline_adjoint_dM"] = {"kernel": "adj_gemm_dM", "bound": "tensor", "achieved": achieved,
                                          "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                          "frac": achieved / peaks["bf16_tflops"], "launches": nl,
                                          "ms": tot, "peak_source": f"bf16 {src}"}
    if args.workload == "full":
        cfg["parts_ms"] = {}
        for name, f in parts.items():
            torch.cuda.synchronize(dev)
            e0.record(st)
            for _ in range(args.steps):
                f()
            e1.record(st)
            torch.cuda.synchronize(dev)
            cfg["parts_ms"][name] = e0.elapsed_time(e1) / args.steps
        _, info = mg.gram_solve(S, gp, handle=h, raise_if_not_pd=False)
        assert int(info.item()) == 0
    # the direct form is FP64 throughout unless its Gamma' update runs on the tensor cores
    dtype = (("f64+bf16x(ozaki)" if args.direct_tensor else "f64") if args.workload == "direct"
             else DTYPE[prec_name])
    print(json.dumps({"metric": METRIC, "value": slices / (ms * 1e-3), "unit": unit,
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": dtype, "data": "synthetic",
                      "config": cfg}), flush=True)


def profiled(h, fn, dev):
    """Per-kernel launches and device time (ms) of one call of fn, from the
    library's own CUDA-event profiler."""
    import ctypes
    import torch
    import paper_1503_08809_gb300 as mg
    lib = mg.lib()
    names = ctypes.create_string_buffer(32 * 64)
    launches = (ctypes.c_int64 * 64)()
    tms = (ctypes.c_double * 64)()
    nout = ctypes.c_int32()
    lib.modal_profile_enable(h.ptr, 1)
    lib.modal_profile_read(h.ptr, 64, names, launches, tms, ctypes.byref(nout))  # reset
    fn()
    torch.cuda.synchronize(dev)
    lib.modal_profile_read(h.ptr, 64, names, launches, tms, ctypes.byref(nout))
    lib.modal_profile_enable(h.ptr, 0)
    out = {}
    for i in range(nout.value):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
        out[nm] = (int(launches[i]), float(tms[i]))
    return out


def fp64_sequential(probs, dps, batched_value, dev, h, n_pts: int = 2):
    """The same models as 64 sequential plain FP64 calls (modal_project_separable,
    MODAL_PREC_FP64), each timed on its first ``n_pts`` radial points (after a
    warm-up call) and scaled by its radial point count -- the FP64 path's time
    is linear in the number of slices; the per-call tables (GL nodes, Legendre
    table) are inside every timed call."""
    import torch
    import paper_1503_08809_gb300 as mg
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms, sampled = 0.0, 0
    for P, dp in zip(probs, dps):
        sub = mg.shard_problem(dp, 0, max(1, P.n_x // n_pts))      # the first ~n_pts radial points
        mg.project_separable(sub, precision=PREC["fp64"], handle=h)
        torch.cuda.synchronize(dev)
        e0.record(st)
        mg.project_separable(sub, precision=PREC["fp64"], handle=h)
        e1.record(st)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1) * P.n_x / sub.n_x
        sampled += sub.n_x * P.n_mu
    slices = sum(P.slices for P in probs)
    value = slices / (total_ms * 1e-3)
    return {"value": value, "unit": "slices/s", "ms_extrapolated": total_ms,
            "sample": f"each of the {len(probs)} models on its first ~{n_pts} radial points "
                      f"({sampled} slices timed), scaled by its radial point count",
            "speedup_of_batched": batched_value / value}


INTEGRATOR_NX = (27, 54, 108, 216, 432, 864)
INTEGRATOR_REF_NX = 1768


def run_integrators(args):
    """Accuracy against time of the two radial rules of Section 3.2.4 (the
    analogue of the paper's integrator study): Gamma' of the l_max 1000 /
    16-function problem with x resampled on 27..864 points, each rule, against
    the Hermite rule on 1768 points; relative RMS error (%) of the unit-normalised
    matrix and the device time of each projection (FP64 by default: the
    tensor-core form's 1e-9 would hide the smaller errors)."""
    import torch
    import paper_1503_08809_gb300 as mg
    import synthetic as syn
    dev = torch.device("cuda", 0)
    prec_name = "fp64" if args.precision == "auto" else args.precision
    prec = PREC[prec_name]
    h = mg.Handle(dev)
    st = torch.cuda.current_stream(dev)

    def project(n, kind, warm=False):
        P = syn.make_problem(1000, 16, n)
        dp = mg.DeviceProblem.from_host(P, device=dev, xw_kind=kind, handle=h)
        if warm:  # the largest run first sizes the scratch for all
            mg.project_separable(dp, precision=prec, handle=h)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g = mg.project_separable(dp, precision=prec, handle=h)
        e1.record(st)
        torch.cuda.synchronize(dev)
        if prec == PREC["ozaki"]:
            mg.handle_status(handle=h)
        return g.cpu().numpy(), e0.elapsed_time(e1), P.slices

    def unit_rmse_pct(g, ref):
        # RMS of the difference relative to the RMS of the reference, both
        # unit-normalised: 100 |G/|G|_F - R/|R|_F|_F
        u = lambda a: a / np.sqrt((a ** 2).sum())
        return 100.0 * float(np.sqrt(((u(g) - u(ref)) ** 2).sum()))

    ref, ref_ms, ref_slices = project(INTEGRATOR_REF_NX, mg.XW_HERMITE, warm=True)
    table = {"trapezium": {}, "hermite": {}}
    tot_ms, tot_slices = ref_ms, ref_slices
    for name, kind in (("trapezium", mg.XW_TRAPEZOID), ("hermite", mg.XW_HERMITE)):
        for n in INTEGRATOR_NX:
            g, ms, sl = project(n, kind)
            table[name][str(n)] = {"rel_rms_pct": unit_rmse_pct(g, ref), "ms": ms}
            tot_ms += ms
            tot_slices += sl
    cfg = {"workload": "lmax1000_nb16_integrators", "l_max": 1000, "nb": 16,
           "n_x": list(INTEGRATOR_NX), "reference": f"hermite rule, {INTEGRATOR_REF_NX} x",
           "precision": prec_name,
           "error": "relative RMS error (%) of the unit-normalised Gamma': 100 |G/|G| - R/|R||_F",
           "study": table, "reference_ms": ref_ms}
    print(json.dumps({"metric": METRIC, "value": tot_slices / (tot_ms * 1e-3), "unit": "slices/s",
                      "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": tot_ms,
                      "higher_is_better": True, "dtype": DTYPE[prec_name], "data": "synthetic",
                      "config": cfg}), flush=True)


def main():
    args = parse()
    if args.workload == "integrators" and args.impl == "ours":
        run_integrators(args)
        return
    if args.workload == "sparse" and args.impl == "ours":
        run_sparse(args)
        return
    if args.workload != "planck" and args.impl == "ours":
        run_extra(args)
        return
    if args.once:
        run_once(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
