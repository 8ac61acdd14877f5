#!/usr/bin/env python3
"""Benchmark of the compressed PMCHWT product on one GB300 (replicas for N > 1).

Workload: lossy dielectric sphere, icosahedral mesh with 20480 triangles
(30720 RWG edges, 61440 unknowns), k0 a = 10, eps_r = 3.2 - 1.9j, cluster leaf
64, admissibility eta = 2, ACA tolerance 1e-4; complex64 operator.  A step is
one product y = Z x with x already resident in HBM; the operator (about 3 GB)
is far larger than L2, so every step streams it from HBM (no flush needed).

Reported beside the headline value:
  roofline      dominant kernel's algorithmic bytes / its mean CUDA-event time,
                against the measured HBM copy bandwidth;
  e2e           the same product through the C interface with host buffers
                (pinned H2D of x and D2H of y inside the timed region);
  fp64_baseline the same product with the complex128 operator (plain FP64 GPU
                form), and both products' error against the float64 oracle on
                sampled rows of the dense product;
  cpu_baseline  the oracle's on-the-fly dense rows, timed on the host cores;
  large         the 602,208-unknown lossy slab (10 x 10 x 1 wavelengths): products
                with complex64 and with BF16 factors, their error on oracle rows,
                a BF16-inner solve refined in FP64, and the 1/8-scale copy's
                currents and absorbed power density against the stored oracle
                solution;
  multi_mesh    16 spheres of uneven size: one product each per step, as separate
                calls, as one CUDA-graph launch, and after autotuning;
  layered       a coated lossy sphere (two surfaces, three regions, 19,200
                unknowns): product and adjoint product of the region-by-region
                operator, a solve against the stored dense oracle solution and the
                coated-sphere series, and the absorbed-power gradient with respect
                to the weights of 64 plane waves;
  planar        the paper's own 2-D operators: dense FP64 Galerkin S, D, N on the
                ellipse of its rank study (aspect 1.5, perimeter 2 pi) at k0 = 64
                and 128 (18 unknowns per wavelength).
`--impl reference` times the oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "compressed BEM matvecs/s and HBM GB/s at 61k/200k unknowns; mixed vs FP64 at 1e-4 err"
UNIT = "matvecs/s"
K0, EPS, LEAF, ETA, ACA_TOL = 10.0, 3.2 - 1.9j, 64, 2.0, 1e-4
LEVEL = 5          # icosphere refinement: 20 * 4**LEVEL triangles (5 -> 20480)
FALLBACK_HBM_GBS = 6800.0


# the large workload: closed lossy slab 10 x 10 x 1 free-space wavelengths (k0 = 2 pi),
# 204 x 204 x 21 face divisions: 200,736 triangles, 301,104 RWG edges, 602,208 unknowns
SLAB = (10.0, 10.0, 1.0, 204, 204, 21)
SLAB_K0 = 2.0 * math.pi
SLAB_NAME = "slab-10x10x1lambda-204x204x21-200736tri-602208unk-k0=2pi-eps3.2-1.9j-leaf64-eta2-aca1e-4"


def workload_name(level):
    nt = 20 * 4 ** level
    return f"sphere-ico{level}-{nt}tri-{3 * nt}unk-k0a10-eps3.2-1.9j-leaf64-eta2-aca1e-4"


def config_dict(extra=None):
    nt = 20 * 4 ** LEVEL
    d = {"workload": workload_name(LEVEL), "unknowns": 3 * nt, "triangles": nt, "rwg_edges": 3 * nt // 2, "k0a": K0,
         "eps_r": [EPS.real, EPS.imag], "leaf_size": LEAF, "eta": ETA, "aca_tol": ACA_TOL, "nrhs": 1,
         "l2": "operator data ~3 GB per product >> 129 MB L2; no flush needed", "parallelism": "replicas"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------
# oracle timing (host cores)
# ---------------------------------------------------------------------------
def oracle_rows(g, x, rows, threads, k0=K0):
    from oracle import operators as O

    chunks = [rows[i::threads] for i in range(threads) if len(rows[i::threads])]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        parts = list(ex.map(lambda r: (r, O.pmchwt_rows_apply(g, k0, EPS, x, r)), chunks))
    dt = time.perf_counter() - t0
    out = {}
    for r, v in parts:
        for i, val in zip(r, v):
            out[int(i)] = val
    return np.array([out[int(i)] for i in rows]), dt


def sample_rows(ne, count, seed=11):
    return np.random.default_rng(seed).choice(2 * ne, count, replace=False)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid):
        self.samples = []
        self.proc = None
        self.uuid = gpu_uuid

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu=uuid,{self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            self.samples.append((time.perf_counter(), parts[1:]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.samples:
            return None
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        where = "inside timed region"
        if not inside:
            inside = sorted(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))[:3]
            where = "nearest samples (timed region shorter than the sampling period)"

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(s[1][0]) for s in inside if num(s[1][0]) is not None]
        mx = [num(s[1][1]) for s in inside if num(s[1][1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4) if s[1][4 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "where": where}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(name, alg_now):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current
    kernel source: (bytes, note).  A capture of a smaller workload of the same kernel
    (its algorithmic bytes recorded beside it) is scaled by the algorithmic bytes of
    this launch, since traffic grows in proportion to them."""
    src = os.path.join(ROOT, "paper_2310_15644_gb300", "csrc", "matvec.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None, None
    for line in open(p):
        parts = line.split()
        if len(parts) < 4 or parts[0] != name or parts[2] != digest:
            continue
        if parts[3] == workload_name(LEVEL):
            return float(parts[1]), "captured on this workload"
        if len(parts) >= 5:
            return float(parts[1]) * alg_now / float(parts[4]), f"scaled from {parts[3]} by algorithmic bytes"
    return None, None


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def run_native(args, rank, world, dist):
    import torch

    import paper_2310_15644_gb300.bem as B
    import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    v, t = W.icosphere(LEVEL)

    def context(prec, **kw):
        opt = B.bem_default_options()
        opt.precision = prec
        opt.leaf_size = LEAF
        opt.eta = ETA
        opt.aca_tol = ACA_TOL
        for key, val in kw.items():
            setattr(opt, key, val)
        h = B.bem_create(opt)
        B.bem_set_mesh(h, v, t)
        B.bem_set_media(h, K0, EPS)
        t0 = time.perf_counter()
        B.bem_assemble(h, sp)
        torch.cuda.synchronize(dev)
        return h, (time.perf_counter() - t0) * 1e3

    def barrier():
        if dist is not None:
            dist.barrier()

    def time_steps(h, xd, yd, dtype, K, W_, profile):
        for _ in range(W_):
            B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dtype, sp)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if profile:
            B.bem_profile_begin(h)
        w0 = time.perf_counter()
        e0.record(stream)
        for _ in range(K):
            B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dtype, sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
        barrier()
        torch.cuda.synchronize(dev)
        prof = B.bem_profile_end(h) if profile else None
        return e0.elapsed_time(e1), (w0, w1), prof

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", "")[:8]
    except Exception:
        pass
    h64, asm64_ms = context(B.BEM_PREC_C64)
    stats = B.bem_stats_get(h64)
    n = B.bem_num_unknowns(h64)
    x = W.complex_normal(n, seed=0).astype(np.complex64)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty_like(xd)
    clocks = ClockSampler(uuid)
    clocks.start()
    ms, (w0, w1), (kms, kcnt) = time_steps(h64, xd, yd, B.BEM_C64, args.steps, args.warmup, True)
    clocks.stop()
    clk = clocks.summary(w0, w1)
    y64 = yd.cpu().numpy().astype(np.complex128)

    # whole job: max over ranks
    t_ms = ms
    if dist is not None:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    ms_per_step = t_ms / args.steps
    value = world * args.steps / (t_ms / 1e3)

    # roofline of the dominant kernel
    peak, peak_kind = measured_peak()
    # FMA peaks of this GPU (our own microbenchmark; no clock or power change)
    fma_peaks = {"fp32_tflops": round(B.bem_measure_fma_peak(False, sp), 2),
                 "fp64_tflops": round(B.bem_measure_fma_peak(True, sp), 3),
                 "source": "bem_measure_fma_peak: 8 independent FMA chains per thread, 8 CTAs of 256 per SM"}
    kb = stats["kernel_bytes_c64"]
    names = B.KERNEL_NAMES
    mean_ms = [kms[i] / max(1, kcnt[i]) for i in range(3)]
    dom = int(np.argmax(mean_ms))
    achieved = kb[dom] / (mean_ms[dom] * 1e-3) / 1e9
    traffic, traffic_note = kernel_traffic(names[dom], kb[dom])
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": round(traffic) if traffic else None, "traffic_source": traffic_note,
                "peak_source": f"{peak_kind} HBM copy bandwidth",
                "algorithmic_bytes_per_launch": int(kb[dom]), "mean_launch_ms": round(mean_ms[dom], 5),
                "kernels": {names[i]: {"mean_ms": round(mean_ms[i], 5), "launches": int(kcnt[i]),
                                       "algorithmic_bytes": int(kb[i]),
                                       "GBps": round(kb[i] / (mean_ms[i] * 1e-3) / 1e9, 1) if mean_ms[i] > 0 else None,
                                       "share": round(kms[i] / max(1e-9, sum(kms)), 4)} for i in range(3)}}
    step_gbs = stats["matvec_bytes_c64"] / (ms_per_step * 1e-3) / 1e9

    # end to end through the C interface with host buffers
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xe = torch.empty_like(xd)
    ye = torch.empty_like(xd)
    for _ in range(args.warmup):
        xe.copy_(xh, non_blocking=True)
        B.bem_matvec(h64, xe.data_ptr(), ye.data_ptr(), 1, B.BEM_C64, sp)
        yh.copy_(ye, non_blocking=True)
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        xe.copy_(xh, non_blocking=True)
        B.bem_matvec(h64, xe.data_ptr(), ye.data_ptr(), 1, B.BEM_C64, sp)
        yh.copy_(ye, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    if dist is not None:
        tt = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e = {"value": round(world * args.steps / (e2e_ms / 1e3), 2), "unit": UNIT,
           "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
           "d2h_bytes_per_step": int(yh.numel() * yh.element_size())}
    # batched right-hand sides: the CUDA-core forms stream the operator once per chunk
    # of 8 vectors, the tensor-core form (BEM_C64_TC) once per pass of 64
    batched = {}
    entry_bytes = stats["matvec_bytes_c64"] - 8 * 2 * n  # entries only (vectors excluded)
    for label, dtype, nrhs, chunk in (("cuda_cores_8", B.BEM_C64, 8, 8), ("cuda_cores_64", B.BEM_C64, 64, 8),
                                      ("tensor_cores_64", B.BEM_C64_TC, 64, 64),
                                      ("tensor_cores_128", B.BEM_C64_TC, 128, 64)):
        X = W.complex_normal(n, seed=3, nrhs=nrhs).astype(np.complex64)
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)
        Yd = torch.empty_like(Xd)
        kb_ = max(3, args.steps // (2 * nrhs))
        for _ in range(3):
            B.bem_matvec(h64, Xd.data_ptr(), Yd.data_ptr(), nrhs, dtype, sp)
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        B.bem_profile_begin(h64)
        e0.record(stream)
        for _ in range(kb_):
            B.bem_matvec(h64, Xd.data_ptr(), Yd.data_ptr(), nrhs, dtype, sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        bms = e0.elapsed_time(e1) / kb_
        pk_ms, pk_cnt = B.bem_profile_end(h64)
        passes = (nrhs + chunk - 1) // chunk
        byt = passes * entry_bytes + 8 * 2 * n * nrhs * 2   # operator once per pass, x read and y written once
        rec = {"matvecs_per_s": round(world * nrhs / (bms / 1e3), 1), "ms_per_call": round(bms, 4),
               "calls": kb_, "operator_passes": passes,
               "hbm_gbps_algorithmic": round(byt / (bms * 1e-3) / 1e9, 1),
               "hbm_frac_of_peak": round(byt / (bms * 1e-3) / 1e9 / peak, 4),
               "kernel_ms_per_pass": {B.KERNEL_NAMES[i]: round(pk_ms[i] / max(1, pk_cnt[i]), 4) for i in range(3)}}
        if dtype == B.BEM_C64_TC:
            kbt = stats["kernel_bytes_tc"]
            rec["kernel_gbps_algorithmic"] = {
                B.KERNEL_NAMES[i]: round(kbt[i] / (pk_ms[i] / max(1, pk_cnt[i]) * 1e-3) / 1e9, 1)
                for i in range(3) if pk_ms[i] > 0}
            rec["t_bytes_per_pass"] = int(8 * stats["t_rows"] * 64)
            ref8 = torch.empty_like(Xd[:8])
            B.bem_matvec(h64, Xd[:8].data_ptr(), ref8.data_ptr(), 8, B.BEM_C64, sp)
            torch.cuda.synchronize(dev)
            d = (Yd[:8] - ref8).abs().max().item() / ref8.abs().max().item()
            rec["max_abs_diff_vs_cuda_cores_rel"] = d
        batched[label] = rec
    B.bem_destroy(h64)

    out = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "complex64 (fp32)", "data": "synthetic",
           "config": config_dict(), "hbm_gbps_algorithmic": round(step_gbs, 1),
           "hbm_frac_of_peak": round(step_gbs / peak, 4), "roofline": roofline, "e2e": e2e,
           "gpu_launches": int(sum(kcnt)), "clocks": clk, "batched_rhs": batched, "measured_fma_peaks": fma_peaks,
           "assembly": {"ms": round(asm64_ms, 1), "near_entries_per_op": stats["near_entries"],
                        "factor_entries": stats["factor_entries"], "max_rank": stats["max_rank"],
                        "far_blocks": stats["n_far"], "far_blocks_dense": stats["n_far_dense"],
                        "near_blocks": stats["n_near"], "bytes_per_product": stats["matvec_bytes_c64"]}}

    if rank == 0 and world == 1:
        g = None
        rows = None
        if not args.no_fp64 or not args.no_cpu_baseline:
            from oracle import rwg

            g = rwg.build(v, t)
            rows = sample_rows(g.ne, max(args.cpu_rows, os.cpu_count() or 1))
        def solve(h, label):
            bd = torch.empty(n, dtype=torch.complex128, device=dev)
            B.bem_rhs_planewave(h, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0], bd.data_ptr(), B.BEM_C128, sp)
            xs = torch.zeros_like(bd)
            warm_solve(h, n, 1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            it, rel, status = B.bem_solve(h, bd.data_ptr(), xs.data_ptr(), 1, sp, raise_on_noconv=False)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            pa, pe, ps = B.bem_power(h, xs.data_ptr(), bd.data_ptr(), 1, sp)
            return {"form": label, "seconds": round(dt, 3), "solves_per_s": round(1.0 / dt, 3), "iterations": it,
                    "ms_per_iteration": round(dt * 1e3 / max(1, it), 4),
                    "relative_residual": float(rel[0]), "converged": status == 0,
                    "Q_abs": pa[0] / np.pi, "Q_ext": pe[0] / np.pi, "Q_sca": ps[0] / np.pi}

        solves = []
        if not args.no_fp64:
            # complex64 GMRES to 1e-6
            opt_s = dict(maxit=3000, gmres_restart=80)
            hs, _ = context(B.BEM_PREC_C64, **opt_s)
            solves.append(solve(hs, "complex64 GMRES, tol 1e-6"))
            # GMRES overhead: time per iteration over the time of one product (restart products included)
            solves[-1]["per_iteration_over_product"] = round(solves[-1]["ms_per_iteration"] / ms_per_step, 3)
            if not args.no_batched_solve:
                out["batched_solve"] = run_batched_solve(dev, stream, B, W, hs,
                                                         batched["tensor_cores_64"]["ms_per_call"])
            B.bem_destroy(hs)
            h128, asm128_ms = context(B.BEM_PREC_C128)
            s128 = B.bem_stats_get(h128)
            xd2 = torch.from_numpy(x.astype(np.complex128)).to(dev)
            yd2 = torch.empty_like(xd2)
            k128 = max(3, args.steps // 8)
            ms2, _, _ = time_steps(h128, xd2, yd2, B.BEM_C128, k128, max(3, args.warmup // 4), False)
            y128 = yd2.cpu().numpy()
            # FP64 arithmetic of the complex128 product: one complex multiply-add (8 FLOP)
            # per stored complex entry (16 bytes)
            fp64_tf = 8.0 * (s128["matvec_bytes_c128"] / 16.0) / (ms2 / k128 * 1e-3) / 1e12
            out["fp64_baseline"] = {"value": round(k128 / (ms2 / 1e3), 2), "unit": UNIT,
                                    "fp64_tflops": round(fp64_tf, 3),
                                    "fp64_frac_of_measured_fma_peak": round(fp64_tf / fma_peaks["fp64_tflops"], 4),
                                    "ms_per_step": round(ms2 / k128, 4), "steps": k128, "dtype": "complex128 (fp64)",
                                    "assembly_ms": round(asm128_ms, 1),
                                    "hbm_gbps_algorithmic": round(s128["matvec_bytes_c128"] / (ms2 / k128 * 1e-3) / 1e9, 1),
                                    "complex64_speedup": round((ms2 / k128) / ms_per_step, 2)}
            B.bem_destroy(h128)
            hs, _ = context(B.BEM_PREC_C128, **opt_s)
            solves.append(solve(hs, "complex128 GMRES, tol 1e-6 (plain FP64 GPU form)"))
            B.bem_destroy(hs)
            hs, _ = context(B.BEM_PREC_C64 | B.BEM_PREC_C128, tol=1e-4, refine_tol=1e-8, **opt_s)
            solves.append(solve(hs, "complex64 GMRES (tol 1e-4) inside FP64 refinement to 1e-8"))
            B.bem_destroy(hs)
            out["solve"] = solves
        if not args.no_calderon:
            out["calderon"] = run_calderon(args, dev, stream, B, W)
        if not args.no_cpu_baseline:
            threads = os.cpu_count() or 1           # every host core (nproc); rows >= threads
            ref, dt = oracle_rows(g, x.astype(np.complex128), rows, threads)
            scale = float(np.sqrt(np.mean(np.abs(y64) ** 2)))
            out["rel_err_vs_oracle"] = float(np.abs(y64[rows] - ref).max() / scale)
            if "fp64_baseline" in out:
                out["fp64_baseline"]["rel_err_vs_oracle"] = float(np.abs(y128[rows] - ref).max() / scale)
            if "batched_solve" in out:
                bs = out["batched_solve"]
                Xh, bh = bs.pop("_x"), bs.pop("_b")
                rows_b = sample_rows(g.ne, 2 * threads, seed=12)
                zx, _ = oracle_rows(g, Xh, rows_b, threads)
                res = np.abs(bh[rows_b] - zx).max(axis=0) / np.sqrt(np.mean(np.abs(bh) ** 2, axis=0))
                from oracle import mie

                q = mie.efficiencies_eps(K0, EPS)
                bs["oracle_check"] = {
                    "residual_rows": f"{len(rows_b)} sampled rows of b - Z x, Z the dense float64 PMCHWT rows",
                    "max_row_residual_over_rms_b": [float(v_) for v_ in res],
                    "mie": {"Q_abs": q["abs"], "Q_ext": q["ext"]},
                    "Q_abs_rel_err_vs_mie": [abs(v_ - q["abs"]) / q["abs"] for v_ in bs["Q_abs"]],
                    "Q_ext_rel_err_vs_mie": [abs(v_ - q["ext"]) / q["ext"] for v_ in bs["Q_ext"]]}
            out["cpu_baseline"] = {"value": round(len(rows) / dt / (2 * g.ne), 6), "unit": UNIT, "cores": threads,
                                   "kind": "oracle",
                                   "sample": f"{len(rows)} of {2 * g.ne} rows of the dense float64 PMCHWT product, "
                                             f"evaluated on the fly (numpy, {threads} threads), {dt:.1f} s",
                                   "error_metric": "max |y_gpu - y_oracle| over sampled rows / rms(y_gpu)"}
        if "batched_solve" in out:
            out["batched_solve"].pop("_x", None)
            out["batched_solve"].pop("_b", None)
        if not args.no_large:
            out["large"] = run_large(args, dev, stream, B, W, peak, not args.no_cpu_baseline)
        if not args.no_multi:
            out["multi_mesh"] = run_multi_mesh(args, dev, stream, B, W)
        if not args.no_layered:
            out["layered"] = run_layered(args, dev, stream, B, W)
        if not args.no_planar:
            out["planar"] = run_planar(args, dev, stream, B, W)
    return out


def warm_solve(h, n, nrhs):
    """A solve of zero right-hand sides: allocates the solver's workspaces (as the
    first solve of a context does) without iterating, so the timed solve that
    follows measures the iterations."""
    import torch

    import paper_2310_15644_gb300.bem as B

    z = torch.zeros((nrhs, n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(z)
    B.bem_solve(h, z.data_ptr(), x.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# batched solves: 64 plane waves on the sphere
# ---------------------------------------------------------------------------
def run_batched_solve(dev, stream, B, W, h, tc_ms):
    """64 plane waves (Fibonacci-sphere directions, seeded random polarisations) on
    the sphere, solved together by the batched GMRES (complex64, tol 1e-6, restart
    80; products on the tensor cores), and 4 of them one at a time for comparison.
    Returns timings, per-wave residuals and efficiencies; the solutions and
    right-hand sides ride along under private keys for the oracle check."""
    import torch

    sp = stream.cuda_stream
    n = 2 * B.bem_num_edges(h)
    nw = 64
    khat, e0 = W.plane_wave_batch(nw, seed=0)
    bd = torch.empty((nw, n), dtype=torch.complex128, device=dev)
    B.bem_rhs_planewave(h, khat, e0, bd.data_ptr(), B.BEM_C128, sp)
    # warm-up: the tensor-core plan and one pass
    xw = torch.zeros((nw, n), dtype=torch.complex64, device=dev)
    yw = torch.empty_like(xw)
    B.bem_matvec(h, xw.data_ptr(), yw.data_ptr(), nw, B.BEM_C64_TC, sp)
    del xw, yw
    xs = torch.zeros_like(bd)
    warm_solve(h, n, nw)
    torch.cuda.synchronize(dev)
    p0 = B.bem_stats_get(h)["tc_passes"]
    t0 = time.perf_counter()
    it, rel, status = B.bem_solve(h, bd.data_ptr(), xs.data_ptr(), nw, sp, raise_on_noconv=False)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    passes = B.bem_stats_get(h)["tc_passes"] - p0
    pa, pe, _ = B.bem_power(h, xs.data_ptr(), bd.data_ptr(), nw, sp, scattered=False)
    # the same waves one at a time (first 4)
    x1 = torch.zeros_like(bd[:4])
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    it1 = 0
    for r in range(4):
        i1, _, _ = B.bem_solve(h, bd[r].data_ptr(), x1[r].data_ptr(), 1, sp, raise_on_noconv=False)
        it1 += i1
    torch.cuda.synchronize(dev)
    dt1 = time.perf_counter() - t1
    d1 = float(((x1 - xs[:4]).abs().pow(2).sum(1).sqrt() / xs[:4].abs().pow(2).sum(1).sqrt()).max().item())
    return {"workload": workload_name(LEVEL), "waves": nw,
            "form": "batched complex64 GMRES(80), tol 1e-6, products on the tensor cores (BEM_C64_TC)",
            "seconds": round(dt, 3), "solves_per_s": round(nw / dt, 2), "converged": status == 0,
            "iterations_total": it, "iterations_mean": round(it / nw, 1),
            "batched_iterations": int(passes),
            "ms_per_batched_iteration": round(dt * 1e3 / max(1, passes), 3),
            "tc_product_ms_64": tc_ms,
            "per_iteration_over_product": round(dt * 1e3 / max(1, passes) / tc_ms, 3),
            "relres_max": float(np.max(rel)), "relres": [float(v) for v in rel],
            "Q_abs": [float(v) / np.pi for v in pa], "Q_ext": [float(v) / np.pi for v in pe],
            "one_at_a_time": {"waves": 4, "seconds": round(dt1, 3), "solves_per_s": round(4 / dt1, 3),
                              "iterations_total": it1, "max_rel_diff_vs_batched": d1},
            "batched_speedup": round((nw / dt) / (4 / dt1), 2),
            "_x": xs.cpu().numpy().T.copy(), "_b": bd.cpu().numpy().T.copy()}


# ---------------------------------------------------------------------------
# large workload: the slab
# ---------------------------------------------------------------------------
def run_large(args, dev, stream, B, W, peak, with_oracle):
    """Products of the 602,208-unknown slab with complex64 and with BF16 factors,
    per-kernel bandwidth, error against oracle rows, and a BF16-inner refined solve
    with its absorbed power; plus the 1/8-scale copy against the stored oracle
    solution (absorbed power and its per-triangle density)."""
    import torch

    sp = stream.cuda_stream
    v, t = W.box_mesh(*SLAB)
    opt = B.bem_default_options()
    opt.precision = B.BEM_PREC_C64 | B.BEM_PREC_BF16F
    opt.leaf_size, opt.eta, opt.aca_tol = LEAF, ETA, ACA_TOL
    opt.tol, opt.refine_tol, opt.maxit, opt.gmres_restart = 1e-3, 1e-6, 5000, 80
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, SLAB_K0, EPS)
    t0 = time.perf_counter()
    B.bem_assemble(h, sp)
    torch.cuda.synchronize(dev)
    asm_ms = (time.perf_counter() - t0) * 1e3
    st = B.bem_stats_get(h)
    n = B.bem_num_unknowns(h)
    x = W.complex_normal(n, seed=0).astype(np.complex64)
    xd = torch.from_numpy(x).to(dev)
    out = {"workload": SLAB_NAME, "unknowns": n, "triangles": len(t),
           "assembly": {"ms": round(asm_ms, 1), "phases_ms": {k: round(val, 1) for k, val in st["assemble_phase_ms"].items()},
                        "near_entries_per_op": st["near_entries"], "factor_entries": st["factor_entries"],
                        "far_blocks": st["n_far"], "far_blocks_split": st["n_far_split"],
                        "blocks_factored": st["n_far_factored"], "far_blocks_dense": st["n_far_dense"],
                        "max_rank": st["max_rank"]}}
    ys = {}
    K = max(10, args.steps // 40)
    for dtype, label, total_key, kern_key in ((B.BEM_C64, "complex64", "matvec_bytes_c64", "kernel_bytes_c64"),
                                              (B.BEM_C64_BF16F, "bf16_factors", "matvec_bytes_bf16f",
                                               "kernel_bytes_bf16f")):
        yd = torch.empty_like(xd)
        for _ in range(3):
            B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dtype, sp)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        B.bem_profile_begin(h)
        e0.record(stream)
        for _ in range(K):
            B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dtype, sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        kms, kcnt = B.bem_profile_end(h)
        ms = e0.elapsed_time(e1) / K
        kb = st[kern_key]
        gbs = st[total_key] / (ms * 1e-3) / 1e9
        out[label] = {"matvecs_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 4), "steps": K,
                      "bytes_per_product": int(st[total_key]), "hbm_gbps_algorithmic": round(gbs, 1),
                      "hbm_frac_of_peak": round(gbs / peak, 4),
                      "kernels": {B.KERNEL_NAMES[i]: {"mean_ms": round(kms[i] / max(1, kcnt[i]), 4),
                                                      "GBps": round(kb[i] / (kms[i] / max(1, kcnt[i]) * 1e-3) / 1e9, 1)
                                                      if kms[i] > 0 else None} for i in range(3)}}
        ys[label] = yd.cpu().numpy().astype(np.complex128)
        # the same product after bem_autotune picked the rows-kernel schedule
        chosen, _ = B.bem_autotune(h, dtype, sp)
        e0.record(stream)
        for _ in range(K):
            B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dtype, sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_t = e0.elapsed_time(e1) / K
        out[label]["autotuned"] = {"slots_per_sm": chosen // 152, "ms_per_step": round(ms_t, 4),
                                   "matvecs_per_s": round(1e3 / ms_t, 2),
                                   "hbm_gbps_algorithmic": round(st[total_key] / (ms_t * 1e-3) / 1e9, 1)}
    if with_oracle:
        from oracle import rwg

        g = rwg.build(v, t)
        rows = sample_rows(g.ne, 16)
        ref, dt = oracle_rows(g, x.astype(np.complex128), rows, os.cpu_count() or 1, k0=SLAB_K0)
        for label, y in ys.items():
            scale = float(np.sqrt(np.mean(np.abs(y) ** 2)))
            out[label]["rel_err_vs_oracle"] = float(np.abs(y[rows] - ref).max() / scale)
        out["oracle_rows"] = {"rows": len(rows), "seconds": round(dt, 1)}
    # solve: BF16-factor GMRES (tol 1e-3 per step) inside FP64 refinement on the complex64 operator
    bd = torch.empty(n, dtype=torch.complex128, device=dev)
    B.bem_rhs_planewave(h, [0.0, 0.0, -1.0], [1.0, 0.0, 0.0], bd.data_ptr(), B.BEM_C128, sp)
    xs = torch.zeros_like(bd)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    it, relres, status = B.bem_solve(h, bd.data_ptr(), xs.data_ptr(), 1, sp, raise_on_noconv=False)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    pa, pe, ps = B.bem_power(h, xs.data_ptr(), bd.data_ptr(), 1, sp)
    out["solve"] = {"form": "BF16-factor GMRES (tol 1e-3) inside FP64 refinement to 1e-6 (complex64 operator)",
                    "seconds": round(dt, 3), "iterations": it, "relative_residual": float(relres[0]),
                    "converged": status == 0, "p_abs": pa[0], "p_ext": pe[0], "p_sca": ps[0]}
    B.bem_destroy(h)
    # the 1/8-scale copy against the stored oracle solution
    gold = os.path.join(ROOT, "tests", "golden", "slab_eighth_oracle.npz")
    if os.path.exists(gold):
        d = np.load(gold)
        dims = [float(a) if i < 3 else int(a) for i, a in enumerate(d["dims"])]
        v8, t8 = W.box_mesh(*dims)
        res8 = {"mesh": "1/8-scale slab 1.25x1.25x1 lambda, 26x26x21, %d unknowns" % d["x"].shape[0]}
        for aca in (1e-4, 1e-5):
            o8 = B.bem_default_options()
            o8.precision = B.BEM_PREC_C64 | B.BEM_PREC_BF16F
            o8.leaf_size, o8.eta, o8.aca_tol = LEAF, ETA, aca
            o8.tol, o8.refine_tol, o8.maxit = 1e-3, 1e-9, 5000
            h8 = B.bem_create(o8)
            B.bem_set_mesh(h8, v8, t8)
            B.bem_set_media(h8, float(d["k0"]), complex(d["eps_r"]))
            B.bem_assemble(h8, sp)
            n8 = B.bem_num_unknowns(h8)
            b8 = torch.empty(n8, dtype=torch.complex128, device=dev)
            B.bem_rhs_planewave(h8, d["khat"].tolist(), d["e0"].tolist(), b8.data_ptr(), B.BEM_C128, sp)
            x8 = torch.zeros_like(b8)
            t0 = time.perf_counter()
            it8, rr8, s8 = B.bem_solve(h8, b8.data_ptr(), x8.data_ptr(), 1, sp, raise_on_noconv=False)
            torch.cuda.synchronize(dev)
            dt8 = time.perf_counter() - t0
            pa8, pe8, _ = B.bem_power(h8, x8.data_ptr(), b8.data_ptr(), 1, sp)
            dens = torch.empty(len(t8), dtype=torch.float64, device=dev)
            B.bem_power_density(h8, x8.data_ptr(), dens.data_ptr(), sp)
            torch.cuda.synchronize(dev)
            xh8 = x8.cpu().numpy()
            ne8 = n8 // 2
            relv = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
            res8[f"aca{aca:g}"] = {"seconds": round(dt8, 3), "iterations": it8, "relative_residual": float(rr8[0]),
                                   "err_J": relv(xh8[:ne8], d["x"][:ne8]), "err_M": relv(xh8[ne8:], d["x"][ne8:]),
                                   "err_p_abs": abs(pa8[0] - float(d["p_abs"])) / abs(float(d["p_abs"])),
                                   "err_density": relv(dens.cpu().numpy(), d["density"])}
            B.bem_destroy(h8)
        out["eighth_scale_vs_oracle"] = res8
    return out


# ---------------------------------------------------------------------------
# layered body: the coated sphere of the gradient workload
# ---------------------------------------------------------------------------
COATED = (4, 1.0, 3, 0.5)          # outer icosphere level and radius, inner level and radius
COATED_K0 = 6.0
COATED_EPS = [1.0, 3.2 - 1.9j, 2.5 - 1.2j]   # exterior (ignored), coating, core


def run_layered(args, dev, stream, B, W):
    """Coated lossy sphere (5,120 + 1,280 triangles, 19,200 unknowns, k0 a = 6): the
    product of the region-by-region operator (three single-medium operators), its
    adjoint, a mixed-precision solve against the stored dense oracle solution and
    the coated-sphere series, and the gradient of the absorbed power with respect
    to the weights of 64 plane waves (w ~ CN(0, 1/64), seed 2)."""
    import torch

    sp = stream.cuda_stream
    v, t, regions = W.coated_sphere(*COATED)
    opt = B.bem_default_options()
    opt.precision = B.BEM_PREC_C64
    opt.leaf_size, opt.eta, opt.aca_tol = LEAF, ETA, ACA_TOL
    opt.tol, opt.maxit = 1e-6, 4000
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_regions(h, COATED_K0, COATED_EPS, regions)
    t0 = time.perf_counter()
    B.bem_assemble(h, sp)
    torch.cuda.synchronize(dev)
    asm = time.perf_counter() - t0
    st = B.bem_stats_get(h)
    n = B.bem_num_unknowns(h)
    out = {"workload": "coated-sphere-ico4r1-ico3r0.5-6400tri-19200unk-k0a6-shell3.2-1.9j-core2.5-1.2j-"
                       "leaf64-eta2-aca1e-4",
           "unknowns": n, "regions": 3, "assembly_ms": round(asm * 1e3, 1),
           "bytes_per_product": st["matvec_bytes_c64"], "max_rank": st["max_rank"]}
    x = torch.from_numpy(W.complex_normal(n, seed=0).astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    K = max(20, args.steps // 10)
    for adj in (False, True):
        f = B.bem_matvec_adjoint if adj else B.bem_matvec
        for _ in range(3):
            f(h, x.data_ptr(), y.data_ptr(), 1, B.BEM_C64, sp)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            f(h, x.data_ptr(), y.data_ptr(), 1, B.BEM_C64, sp)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / K
        out["adjoint_product" if adj else "product"] = {
            "ms": round(ms, 4), "matvecs_per_s": round(1e3 / ms, 1),
            "hbm_gbps_algorithmic": round(st["matvec_bytes_c64"] / (ms * 1e-3) / 1e9, 1), "steps": K}
    gold = os.path.join(ROOT, "tests", "golden", "coated_sphere_oracle.npz")
    if os.path.exists(gold):
        d = np.load(gold)
        b = torch.empty(n, dtype=torch.complex128, device=dev)
        B.bem_rhs_planewave(h, d["khat"].tolist(), d["e0"].tolist(), b.data_ptr(), B.BEM_C128, sp)
        xs = torch.zeros_like(b)
        warm_solve(h, n, 1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        it, relres, status = B.bem_solve(h, b.data_ptr(), xs.data_ptr(), 1, sp, raise_on_noconv=False)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        pa, pe, ps = B.bem_power(h, xs.data_ptr(), b.data_ptr(), 1, sp)
        xh = xs.cpu().numpy()
        ne = n // 2
        relv = lambda a, c: float(np.linalg.norm(a - c) / np.linalg.norm(c))  # noqa: E731
        area = math.pi * COATED[1] ** 2
        q = {"ext": pe[0] / area, "abs": pa[0] / area, "sca": ps[0] / area}
        series = dict(zip(("ext", "abs", "sca"), d["mie"].tolist()))
        oracle = {"ext": float(d["p_ext"]) / area, "abs": float(d["p_abs"]) / area, "sca": float(d["p_sca"]) / area}
        out["solve"] = {"form": "complex64 GMRES(50) to 1e-6, ACA 1e-4", "seconds": round(dt, 3), "iterations": it,
                        "relative_residual": float(relres[0]), "converged": status == 0,
                        "err_J_vs_dense_oracle": relv(xh[:ne], d["x"][:ne]),
                        "err_M_vs_dense_oracle": relv(xh[ne:], d["x"][ne:]),
                        "Q": {k: round(q[k], 6) for k in q},
                        "Q_dense_oracle": {k: round(oracle[k], 6) for k in oracle},
                        "Q_coated_sphere_series": {k: round(series[k], 6) for k in series}}
    kh, e0 = W.plane_wave_batch(64, seed=0)
    bm = torch.empty(64, n, dtype=torch.complex128, device=dev)
    B.bem_rhs_planewave(h, kh, e0, bm.data_ptr(), B.BEM_C128, sp)
    w = W.complex_normal(64, seed=2) / 8.0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    p, grad, itg = B.bem_grad_weights(h, bm.data_ptr(), w, stream=sp)
    torch.cuda.synchronize(dev)
    out["weight_gradient"] = {"plane_waves": 64, "seconds": round(time.perf_counter() - t0, 3),
                              "iterations_forward_plus_adjoint": itg, "p_abs": p,
                              "grad_norm": float(np.linalg.norm(grad))}
    B.bem_destroy(h)
    return out


# ---------------------------------------------------------------------------
# Calderon-preconditioned PMCHWT: iterations under refinement
# ---------------------------------------------------------------------------
def calderon_batched(dev, sp, B, W, h, n, nw=64):
    """The 64 plane waves of the batched-solve workload through the preconditioned
    batched GMRES (tensor-core products of both operators)."""
    import torch

    khat, e0 = W.plane_wave_batch(nw, seed=0)
    bw = torch.empty((nw, n), dtype=torch.complex128, device=dev)
    B.bem_rhs_planewave(h, khat, e0, bw.data_ptr(), B.BEM_C128, sp)
    warm_solve(h, n, nw)
    xw = torch.zeros_like(bw)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    it, rel, st = B.bem_solve(h, bw.data_ptr(), xw.data_ptr(), nw, sp, raise_on_noconv=False)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    pa, _, _ = B.bem_power(h, xw.data_ptr(), bw.data_ptr(), nw, sp, scattered=False)
    return {"waves": nw, "seconds": round(dt, 3), "solves_per_s": round(nw / dt, 2), "converged": st == 0,
            "iterations_mean": round(it / nw, 1), "relres_max": float(np.max(rel)),
            "Q_abs_first4": [float(q) / np.pi for q in pa[:4]]}


def run_calderon(args, dev, stream, B, W, levels=(3, 4, 5), near_only=0, precond_tol=3e-2):
    """Plain and Calderon-preconditioned (BEM_PRECOND_CALDERON) complex64 GMRES on the
    icospheres of the 61k-unknown workload's family (k0 a = 10, eps_r 3.2 - 1.9j,
    plane wave), both with FP64 residual refinement to 1e-6: iterations, wall time,
    time per iteration and the agreement of the two solutions; at the finest level
    also the device time of one preconditioner application against its algorithmic
    bytes."""
    import torch

    sp = stream.cuda_stream
    rows = []
    for level in levels:
        v, t = W.icosphere(level)
        rec = {"level": level, "triangles": len(t), "unknowns": 3 * len(t)}
        xs = {}
        for label, pre in (("plain", B.BEM_PRECOND_NONE), ("calderon", B.BEM_PRECOND_CALDERON)):
            opt = B.bem_default_options()
            opt.precision = B.BEM_PREC_C64
            opt.leaf_size, opt.eta, opt.aca_tol = LEAF, ETA, ACA_TOL
            opt.maxit, opt.gmres_restart, opt.refine_tol = 3000, 80, 1e-6
            opt.preconditioner = pre
            opt.precond_near_only, opt.precond_aca_tol = near_only, precond_tol
            h = B.bem_create(opt)
            try:
                B.bem_set_mesh(h, v, t)
                B.bem_set_media(h, K0, EPS)
                t0 = time.perf_counter()
                B.bem_assemble(h, sp)
                torch.cuda.synchronize(dev)
                asm = time.perf_counter() - t0
                n = B.bem_num_unknowns(h)
                bd = torch.empty(n, dtype=torch.complex128, device=dev)
                B.bem_rhs_planewave(h, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0], bd.data_ptr(), B.BEM_C128, sp)
                warm_solve(h, n, 1)
                xd = torch.zeros_like(bd)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                it, rel, st = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, sp, raise_on_noconv=False)
                torch.cuda.synchronize(dev)
                dt = time.perf_counter() - t0
                r = {"iterations": it, "seconds": round(dt, 4), "ms_per_iteration": round(dt * 1e3 / max(it, 1), 4),
                     "relative_residual": float(rel[0]), "converged": st == 0, "assembly_s": round(asm, 2)}
                if pre == B.BEM_PRECOND_CALDERON:
                    s = B.bem_stats_get(h)
                    r.update({"refined_unknowns": 2 * s["precond_fine_ne"],
                              "gram_chebyshev_steps": s["precond_gram_steps"],
                              "gram_interval": [round(q, 4) for q in s["precond_gram_interval"]],
                              "preconditioner_assembly_s": round(s["precond_assemble_ms"] / 1e3, 2),
                              "preconditioner_bytes_per_vector": s["precond_bytes_c64"],
                              "operator_bytes_per_vector": s["matvec_bytes_c64"]})
                    if level == max(levels):
                        xa = torch.from_numpy(W.complex_normal(n, seed=4).astype(np.complex64)).to(dev)
                        ya = torch.empty_like(xa)
                        for _ in range(3):
                            B.bem_precond_apply(h, xa.data_ptr(), ya.data_ptr(), 1, B.BEM_C64, sp)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        reps = 20
                        torch.cuda.synchronize(dev)
                        e0.record(stream)
                        for _ in range(reps):
                            B.bem_precond_apply(h, xa.data_ptr(), ya.data_ptr(), 1, B.BEM_C64, sp)
                        e1.record(stream)
                        torch.cuda.synchronize(dev)
                        ms = e0.elapsed_time(e1) / reps
                        r["preconditioner_apply_ms"] = round(ms, 4)
                        r["preconditioner_apply_gbps_algorithmic"] = round(s["precond_bytes_c64"] / (ms * 1e-3) / 1e9, 1)
                        del xa, ya
                        if not getattr(args, "no_batched_solve", False):
                            r["batched_64_waves"] = calderon_batched(dev, sp, B, W, h, n)
                xs[label] = xd.cpu().numpy()
                rec[label] = r
            finally:
                B.bem_destroy(h)
        ne = rec["unknowns"] // 2
        x0, x1 = xs["plain"], xs["calderon"]
        rec["solution_rel_diff_J"] = float(np.linalg.norm(x1[:ne] - x0[:ne]) / np.linalg.norm(x0[:ne]))
        rec["solution_rel_diff_M"] = float(np.linalg.norm(x1[ne:] - x0[ne:]) / np.linalg.norm(x0[ne:]))
        rec["speedup_over_plain"] = round(rec["plain"]["seconds"] / rec["calderon"]["seconds"], 3)
        rows.append(rec)
    return {"workload": f"icospheres, k0 a = {K0}, eps_r {EPS}, plane wave +z; complex64 GMRES(80), FP64 "
                        f"residual refinement to 1e-6; refined operator ACA tol {precond_tol}", "levels": rows}


# ---------------------------------------------------------------------------
# the paper's own two-dimensional operators
# ---------------------------------------------------------------------------
def run_planar(args, dev, stream, B, W):
    """Dense 2-D Galerkin S, D and N on the ellipse of the paper's rank study (aspect
    1.5, perimeter 2 pi, 18 unknowns per wavelength: N = 18 k0), in the FP64 form and
    the FP32 form (well-separated pairs in FP32), with the FP32 form's deviation."""
    import torch

    sp = stream.cuda_stream
    out = {"curve": "ellipse aspect 1.5 perimeter 2pi, N = 18 k0", "cases": []}
    for k0 in (64.0, 128.0):
        n = int(round(18 * k0))
        verts = W.ellipse_polygon(n, 1.5, 2 * math.pi)
        rec = {"k0": k0, "n": n}
        ref = None
        for form, fp32 in (("fp64", False), ("fp32", True)):
            mats = [torch.empty(n, n, dtype=torch.complex128, device=dev) for _ in range(3)]
            call = lambda: B.bem_planar_operators(None, verts, k0, mats[0].data_ptr(),  # noqa: E731
                                                  mats[1].data_ptr(), mats[2].data_ptr(), sp, fp32=fp32)
            call()
            torch.cuda.synchronize(dev)
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                call()
            torch.cuda.synchronize(dev)
            ms = (time.perf_counter() - t0) / reps * 1e3
            rec[form] = {"ms": round(ms, 2), "segment_pairs_per_s": round(n * n / (ms * 1e-3), 1),
                         "finite": bool(all(torch.isfinite(torch.view_as_real(m)).all().item() for m in mats))}
            if ref is None:
                ref = mats
            else:
                # the FP32 form against the FP64 one: max |difference| / max |entry| per operator
                rec[form]["max_dev_vs_fp64"] = [float(((m - r).abs().max() / r.abs().max()).item())
                                                for m, r in zip(mats, ref)]
                del mats
        del ref
        out["cases"].append(rec)
    out["fast_solver"] = run_planar_pipeline(args, dev, stream, B, W)
    return out


def run_planar_pipeline(args, dev, stream, B, W, tol=1e-4):
    """The paper's 2-D fast direct solver on the GPU (Sec. III): C_p of the ellipse and of
    its circular counterpart (Eq. 16), the skeleton of C_p - C_p,c by the randomized
    range finder (Eq. 17, seeded Gaussian test vectors, blocks of 8) and one Woodbury
    solve (Eq. 18), against N = 18 k0, with the operators in FP64 and in the FP32
    form; in the cpu_baseline leg the oracle runs the same stages on the host cores
    for the smallest case."""
    import torch

    sp = stream.cuda_stream
    cases = []
    for k0, fp32 in [(k, f) for f in (False, True) for k in (8.0, 16.0, 32.0, 64.0)]:
        n = int(round(18 * k0))
        verts = W.ellipse_polygon(n, 1.5, 2 * math.pi)
        per = float(np.sum(np.hypot(*(np.roll(verts, -1, axis=0) - verts).T)))
        rad = per / (2 * n * math.sin(math.pi / n))
        th = 2 * math.pi * np.arange(n) / n
        cverts = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
        a = per / (2 * math.pi)
        cp = torch.empty((n, n), dtype=torch.complex128, device=dev)
        cc = torch.empty_like(cp)
        omega = torch.from_numpy(np.ascontiguousarray(W.complex_normal(n, seed=7, nrhs=n).T)).to(dev)
        U = torch.empty_like(cp)
        Vt = torch.empty_like(cp)
        b = torch.from_numpy(W.complex_normal(n, seed=8)).to(dev)
        x = torch.empty_like(b)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        B.bem_planar_calderon(None, verts, k0, cp.data_ptr(), 0, 0, 0.0, sp, fp32=fp32)
        B.bem_planar_calderon(None, cverts, k0, cc.data_ptr(), 0, 0, a, sp, fp32=fp32)
        t1 = time.perf_counter()
        A = cp - cc
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        r = B.bem_planar_skeleton(None, A.data_ptr(), n, omega.data_ptr(), n, tol, 8, U.data_ptr(), Vt.data_ptr(), sp)
        t3 = time.perf_counter()
        cc0 = cc[:, 0].contiguous()
        torch.cuda.synchronize(dev)
        t4 = time.perf_counter()
        B.bem_planar_woodbury_solve(None, cc0.data_ptr(), n, U.data_ptr(), Vt.data_ptr(), r, b.data_ptr(),
                                    x.data_ptr(), 1, sp)
        t5 = time.perf_counter()
        res = (cp @ x - b).abs().pow(2).sum().sqrt().item() / b.abs().pow(2).sum().sqrt().item()
        cases.append({"k0": k0, "n": n, "operators": "fp32 far pairs" if fp32 else "fp64", "skeleton_rank": r,
                      "tol": tol,
                      "calderon_s": round(t1 - t0, 4), "skeleton_s": round(t3 - t2, 4),
                      "woodbury_solve_s": round(t5 - t4, 4), "compression_s": round((t1 - t0) + (t3 - t2), 4),
                      "relative_residual_of_C_p_x": res})
        del cp, cc, A, U, Vt, omega
    out = {"curve": "ellipse aspect 1.5 perimeter 2pi, N = 18 k0", "cases": cases}
    if not args.no_cpu_baseline:
        from oracle import planar as PL

        ocases = []
        for k0 in (8.0,):  # the dense oracle operators take about 7 s here, 30 s at k0 = 16
            n = int(round(18 * k0))
            poly = PL.Polygon(W.ellipse_polygon(n, 1.5, 2 * math.pi))
            t0 = time.perf_counter()
            Cp, _, _ = PL.calderon_cfie(poly, k0)
            Cc, _, _ = PL.calderon_cfie(PL.circular_counterpart(poly), k0, a=PL.curvature_radius(poly))
            U, Vt = PL.skeleton(Cp, Cc, W.complex_normal(n, seed=7, nrhs=n), tol)
            dt = time.perf_counter() - t0
            ocases.append({"k0": k0, "n": n, "compression_s": round(dt, 3), "skeleton_rank": int(U.shape[1])})
        out["oracle_on_host_cores"] = {"cores": os.cpu_count() or 1, "cases": ocases,
                                       "kind": "oracle (numpy, float64)"}
    return out


# ---------------------------------------------------------------------------
# many meshes of uneven size in one graph launch
# ---------------------------------------------------------------------------
def run_multi_mesh(args, dev, stream, B, W, count=16):
    """16 geodesic spheres of uneven size (1280-20480 triangles, random radius, k0
    and eps_r; workloads.uneven_sphere_batch, seed 1): one product of every mesh
    per step, issued as 16 bem_matvec calls on one stream, as one CUDA-graph launch
    (bem_batch_launch), and as one graph launch after bem_autotune of each mesh."""
    import torch

    sp = stream.cuda_stream
    specs = W.uneven_sphere_batch(count, seed=1)
    hs, xs, ys, tris, unk = [], [], [], [], []
    t0 = time.perf_counter()
    for i, sp_ in enumerate(specs):
        v, t = W.geodesic_sphere(sp_["freq"], sp_["radius"])
        opt = B.bem_default_options()
        opt.precision = B.BEM_PREC_C64
        opt.leaf_size, opt.eta, opt.aca_tol = LEAF, ETA, ACA_TOL
        h = B.bem_create(opt)
        B.bem_set_mesh(h, v, t)
        B.bem_set_media(h, sp_["k0"], sp_["eps_r"])
        B.bem_assemble(h, sp)
        n = B.bem_num_unknowns(h)
        hs.append(h)
        xs.append(torch.from_numpy(W.complex_normal(n, seed=100 + i).astype(np.complex64)).to(dev))
        ys.append(torch.empty_like(xs[-1]))
        tris.append(len(t))
        unk.append(n)
    torch.cuda.synchronize(dev)
    asm_s = time.perf_counter() - t0
    K = max(10, args.steps // 20)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / K

    def seq():
        for h, x, y in zip(hs, xs, ys):
            B.bem_matvec(h, x.data_ptr(), y.data_ptr(), 1, B.BEM_C64, sp)

    out = {"meshes": count, "triangles": tris, "unknowns_total": int(sum(unk)), "assembly_s": round(asm_s, 2),
           "steps": K}
    ms_seq = timed(seq)
    batch = B.bem_batch_create(hs, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], [1] * count,
                               B.BEM_C64, sp)
    ms_graph = timed(lambda: B.bem_batch_launch(batch, sp))
    B.bem_batch_destroy(batch)
    chosen = [B.bem_autotune(h, B.BEM_C64, sp)[0] for h in hs]
    batch = B.bem_batch_create(hs, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], [1] * count,
                               B.BEM_C64, sp)
    ms_tuned = timed(lambda: B.bem_batch_launch(batch, sp))
    B.bem_batch_destroy(batch)
    for h in hs:
        B.bem_destroy(h)
    out.update({"ms_per_step_sequential": round(ms_seq, 4), "ms_per_step_graph": round(ms_graph, 4),
                "ms_per_step_graph_autotuned": round(ms_tuned, 4),
                "meshes_per_s_graph_autotuned": round(count / (ms_tuned * 1e-3), 1),
                "autotuned_slots_per_sm": [c // 152 for c in chosen]})
    return out


def run_tc_only(args):
    """Tensor-core product of 64 vectors alone, W warm-up and K timed calls (one
    process, one GPU): the command profiling captures of its kernels run."""
    import torch

    import paper_2310_15644_gb300.bem as B
    import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    v, t = W.icosphere(LEVEL)
    opt = B.bem_default_options()
    opt.precision, opt.leaf_size, opt.eta, opt.aca_tol = B.BEM_PREC_C64, LEAF, ETA, ACA_TOL
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, K0, EPS)
    B.bem_assemble(h, sp)
    n = B.bem_num_unknowns(h)
    X = torch.from_numpy(np.ascontiguousarray(W.complex_normal(n, seed=3, nrhs=64).astype(np.complex64).T)).to(dev)
    Y = torch.empty_like(X)
    for _ in range(args.warmup):
        B.bem_matvec(h, X.data_ptr(), Y.data_ptr(), 64, B.BEM_C64_TC, sp)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        B.bem_matvec(h, X.data_ptr(), Y.data_ptr(), 64, B.BEM_C64_TC, sp)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    B.bem_destroy(h)
    return {"workload": workload_name(LEVEL), "vectors": 64, "ms_per_call": round(ms, 4),
            "matvecs_per_s": round(64 / (ms * 1e-3), 1)}


# ---------------------------------------------------------------------------
# reference arm: the oracle alone on host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    import workloads as W
    from oracle import rwg

    v, t = W.icosphere(LEVEL)
    g = rwg.build(v, t)
    x = W.complex_normal(2 * g.ne, seed=0).astype(np.complex64).astype(np.complex128)
    threads = os.cpu_count() or 1                       # every host core (nproc)
    nrows = threads * max(1, -(-args.ref_rows // threads))  # a whole number of rows per thread
    rng = np.random.default_rng(5)
    for _ in range(args.warmup):
        oracle_rows(g, x, rng.choice(2 * g.ne, nrows, replace=False), threads)
    tot = 0.0
    for _ in range(args.steps):
        _, dt = oracle_rows(g, x, rng.choice(2 * g.ne, nrows, replace=False), threads)
        tot += dt
    value = args.steps * nrows / tot / (2 * g.ne)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "complex128 (fp64)",
            "data": "synthetic",
            "config": config_dict({"reference": "float64 CPU oracle (dense PMCHWT rows on the fly)"}),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: {nrows} random rows of the {2 * g.ne}-row dense product, "
                                       f"one numpy thread per core ({threads})"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-rows", type=int, default=256, help="oracle rows timed for cpu_baseline")
    ap.add_argument("--ref-rows", type=int, default=8, help="oracle rows per step of the reference arm")
    ap.add_argument("--no-fp64", action="store_true", help="skip the complex128 GPU comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing")
    ap.add_argument("--no-large", action="store_true", help="skip the 602,208-unknown slab")
    ap.add_argument("--no-multi", action="store_true", help="skip the 16-mesh graph batch")
    ap.add_argument("--no-layered", action="store_true", help="skip the coated (two-region) sphere")
    ap.add_argument("--no-planar", action="store_true", help="skip the 2-D operator assembly")
    ap.add_argument("--no-batched-solve", action="store_true", help="skip the 64-plane-wave batched solve")
    ap.add_argument("--no-calderon", action="store_true", help="skip the Calderon-preconditioned solves")
    ap.add_argument("--tc-only", action="store_true",
                    help="only the tensor-core product of 64 vectors (profiling captures of its kernels)")
    ap.add_argument("--calderon-only", action="store_true",
                    help="only the plain and Calderon-preconditioned solves at --level (profiling captures)")
    ap.add_argument("--level", type=int, default=5,
                    help="icosphere level (5 = the 61440-unknown workload; smaller levels for profiling captures)")
    args = ap.parse_args()
    global LEVEL
    LEVEL = args.level
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    if args.tc_only:
        out = run_tc_only(args)
    elif args.calderon_only:
        import torch

        import paper_2310_15644_gb300.bem as B
        import workloads as W

        dev = torch.device("cuda", 0)
        out = run_calderon(args, dev, torch.cuda.current_stream(dev), B, W, levels=(LEVEL,))
    else:
        out = run_native(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
