"""Benchmark: full Eyre-Milton solves of a 256^3 three-phase RVE on one GB300 (or N replicas).

One step = voxelize the RVE's sphere list (device-resident) and solve the cell problem
for the three unit gradients to tol 1e-8 (eps_comp and eps_eq), returning K.
Workload: 100 identical non-overlapping spheres at 40 % volume fraction (seeded
RSA + growth sweeps), layer l = 0.3, conductivities 0.20 / 0.25 / 400 (contrast 2000).

value  = voxel-iterations/s = sum over steps of N^3 * (sweeps over the 3 gradients) / time,
         inputs resident in HBM, device time from CUDA events around the K timed steps,
         max over ranks; fields (4.2 GB) are far larger than L2, so no flush is needed.
e2e    = the same metric through the public C ABI with host buffers: the sphere list
         and the phase grid cross host<->device inside every step.
Multi-GPU: independent replicas (one RVE per rank, seed 3000 + rank), weak scaling.

--impl reference times the CPU oracle (the FP64 numpy/scipy implementation written from
the paper) on the host cores, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
N_SPHERES, F_SP, LAYER, SEED = 100, 0.40, 0.3, 3000
K_PHASES = (0.20, 0.25, 400.0)
TOL = 1e-8
METRIC = "voxel-iterations/s at 256^3 (3 unit gradients, tol 1e-8)"
UNIT = "voxel-iter/s"


def workload_config(precision: str) -> dict:
    state_gb = 4.2 * (N_GRID / 256) ** 3    # FP32-bulk state of the three gradients
    return {"workload": f"rsa{N_GRID}: {N_GRID}^3 RVE, 100 spheres at 40% (RSA + growth sweeps), layer 0.3, "
                        "k 0.20/0.25/400 (contrast 2000), tol 1e-8, 3 unit gradients",
            "N": N_GRID, "n_spheres": N_SPHERES, "f_sp": F_SP, "layer": LAYER, "k": list(K_PHASES),
            "tol": TOL, "precision": precision, "seed": SEED,
            "l2": f"inputs larger than L2 (solver fields {state_gb:.1f} GB vs 129 MB L2), no flush"}


def replica_seed(rank: int) -> int:
    """RVE realization of a rank: independent replicas, one RVE per GPU (weak scaling)."""
    return SEED + rank


def job_totals(seconds: float, voxel_iters: float, world: int, device: str = "cuda"):
    """Whole-job totals of an independent-replica run: the slowest rank's time and the sum
    of every rank's voxel-iterations.  These two reductions (and the barriers around the
    timed region) are the only communication; the data path has no collective."""
    if world == 1:
        return seconds, voxel_iters
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    v = torch.tensor([voxel_iters], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def torch_fft_sweep(phase, k, N: int, device):
    """Comparison point (not the product path): one Eyre-Milton sweep in the same tau form,
    tau^{n+1} = (I - 2P)(Y tau^n) + 2 k0 E, written with torch.fft (cuFFT on a GPU) and
    torch pointwise operations in FP32.  Returns sweep(tau, E) for tau of shape (3, N, N, N)."""
    import torch
    kk = torch.tensor(k, dtype=torch.float64)
    k0 = float(torch.sqrt(kk.min() * kk.max()))
    Y = ((kk - k0) / (kk + k0)).to(torch.float32).to(device)[phase.long().reshape(N, N, N)]
    m = torch.fft.fftfreq(N, 1.0 / N).to(device)            # signed modes, -N/2 .. N/2 - 1
    m = torch.where(m == -N // 2, torch.full_like(m, N // 2), m)
    mx = torch.arange(N // 2 + 1, device=device, dtype=m.dtype)
    MZ, MY, MX = torch.meshgrid(m, m, mx, indexing="ij")
    comps = [MX, MY, MZ]
    nonzero = sum((c != 0).to(torch.int32) for c in comps)
    # Nyquist components dropped unless they are the mode's only nonzero component
    d = torch.stack([torch.where((c == N // 2) & (nonzero > 1), torch.zeros_like(c), c) for c in comps]).to(torch.float32)
    n2 = (d * d).sum(0)
    inv = torch.where(n2 > 0, 2.0 / torch.where(n2 > 0, n2, torch.ones_like(n2)), torch.zeros_like(n2))

    def sweep(tau, E):
        S = torch.fft.rfftn(Y * tau, dim=(1, 2, 3))
        dot = (d * S).sum(0)
        S = S - d * (inv * dot)
        S[:, 0, 0, 0] += torch.tensor([2.0 * k0 * e * N ** 3 for e in E], dtype=S.dtype, device=device)
        return torch.fft.irfftn(S, s=(N, N, N), dim=(1, 2, 3))

    return sweep


def k_entry_err(K, Kref, floor_frac: float = 1e-2) -> float:
    """Largest relative error over the entries of K; entries below floor_frac times the
    largest diagonal entry of Kref are compared with that floor."""
    floor = floor_frac * float(np.abs(np.diag(Kref)).max())
    return float((np.abs(np.asarray(K) - Kref) / np.maximum(np.abs(Kref), floor)).max())


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_phase(spheres):
    from oracle import em as om
    return om.voxelize(spheres, LAYER, N_GRID)


def oracle_sample(ph, sweeps: int = 1) -> dict:
    """Time `sweeps` oracle sweeps (steps 2-7) of one gradient on the 256^3 RVE."""
    from oracle import em as om
    t0 = time.perf_counter()
    om.em_solve(ph, K_PHASES, (1.0, 0.0, 0.0), tol=0.0, max_iter=sweeps)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "voxel_iters": sweeps * N_GRID ** 3, "threads": om._workers()}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1504_07499_gb300 import inputs as I
    ph = oracle_phase(I.generate_spheres(SEED, N_SPHERES, F_SP).spheres)
    for _ in range(args.warmup):
        oracle_sample(ph, 1)
    tot_t, tot_v, thr = 0.0, 0, 1
    for _ in range(args.steps):
        r = oracle_sample(ph, 1)
        tot_t += r["seconds"]
        tot_v += r["voxel_iters"]
        thr = r["threads"]
    value = tot_v / tot_t
    sample = "one oracle sweep (steps 2-7, one gradient) of the 256^3 RVE per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config("fp64 (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hmg", choices=["hmg", "reference"])
    ap.add_argument("--precision", default="fp32bulk", choices=["fp32bulk", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-cufft", action="store_true", help="skip the torch.fft (cuFFT) comparison sweeps")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve", "contrast", "schemes", "layers"],
                    help="single: the 256^3 RVE (default); batch: 64 mixed-size RVEs in one engine; "
                         "serve: Poisson request stream through hmg_submit/hmg_poll; "
                         "contrast: the 256^3 RVE over 4 contrasts x 3 layers, FP32 bulk and FP64; "
                         "schemes: Eyre-Milton vs the basic scheme at 3 contrasts; "
                         "layers: the paper's sweep over the coating layer at 64^3/128^3/256^3")
    ap.add_argument("--requests", type=int, default=48, help="serve mode: requests per arrival rate")
    ap.add_argument("--variant", type=int, default=-1,
                    help="pin the FP32 kernel variant of the 256^3 grid (0..63, see hmg_set_variant); "
                         "default: autotuned on the device")
    ap.add_argument("--grid", type=int, default=256, choices=[256, 512],
                    help="single mode: grid size of the RVE (256 is the benchmark workload; 512 the "
                         "largest grid, the same spheres at twice the resolution)")
    ap.add_argument("--sweeps-only", type=int, default=0,
                    help="profiling case: voxelize, run the solve for this many sweeps (max_iter), exit")
    args = ap.parse_args()
    global N_GRID, METRIC
    N_GRID = args.grid
    METRIC = METRIC.replace("256^3", f"{N_GRID}^3")
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "contrast":
        run_contrast(args)
        return
    if args.mode == "schemes":
        run_schemes(args)
        return
    if args.mode == "layers":
        run_layers(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return

    import torch
    import torch.distributed as dist

    from paper_1504_07499_gb300 import build, hmg, inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    prec = hmg.HMG_FP32_BULK if args.precision == "fp32bulk" else hmg.HMG_FP64
    ctx = hmg.Context(local)
    seed = replica_seed(rank)
    sl = I.generate_spheres(seed, N_SPHERES, F_SP)
    sph_d = torch.from_numpy(np.ascontiguousarray(sl.spheres)).cuda()
    phase_d = torch.empty(N_GRID ** 3, dtype=torch.uint8, device="cuda")
    N3 = N_GRID ** 3

    def step():
        hmg.hmg_voxelize(ctx.handle, sph_d, LAYER, N_GRID, phase_d)
        K, info, _ = hmg.hmg_solve(ctx.handle, phase_d, N_GRID, K_PHASES, TOL, prec)
        return K, info

    if args.variant >= 0:
        hmg.hmg_set_variant(ctx.handle, N_GRID, args.variant)
    if args.sweeps_only:
        # profiling case: the first sweeps of the benchmark solve itself (three gradients,
        # chained blocks of FP32 sweeps in the launch configuration of the timed solves)
        hmg.hmg_voxelize(ctx.handle, sph_d, LAYER, N_GRID, phase_d)
        hmg.hmg_solve(ctx.handle, phase_d, N_GRID, K_PHASES, TOL, prec, args.sweeps_only,
                      allow=(hmg.HMG_OK, hmg.HMG_NOT_CONVERGED))
        torch.cuda.synchronize()
        ctx.close()
        return

    for _ in range(args.warmup):
        step()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sweeps, lat, Ks = 0, [], []
    for _ in range(args.steps):
        t = time.perf_counter()
        K_step, info = step()
        lat.append(time.perf_counter() - t)
        sweeps += sum(info["iters"])
        Ks.append(K_step)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    # kernel breakdown from one more solve of the same RVE, outside the timed region, with
    # the library's tracer on (CUDA events on the launching stream around every launch);
    # a solve launches the same kernels every time, so its launch count per step holds
    # for the timed steps too
    hmg.hmg_trace_enable(ctx.handle, True)
    _, info_tr = step()
    hmg.hmg_trace_enable(ctx.handle, False)
    trace = hmg.hmg_trace_read(ctx.handle)
    assert list(info_tr["iters"]) == list(info["iters"]), "traced solve took other sweep counts"

    ms_max, vox_all = job_totals(ms, float(sweeps * N3), world)
    value = vox_all / (ms_max / 1e3)

    # --- end to end through the C ABI with host buffers ---------------------------
    sph_h = torch.from_numpy(np.ascontiguousarray(sl.spheres)).pin_memory().numpy()
    phase_h = torch.empty(N3, dtype=torch.uint8).pin_memory().numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_sweeps = 0
    for _ in range(args.e2e_steps):
        hmg.hmg_voxelize(ctx.handle, sph_h, LAYER, N_GRID, phase_h)               # D2H phase grid
        K, info, _ = hmg.hmg_solve(ctx.handle, phase_h, N_GRID, K_PHASES, TOL, prec)  # H2D phase, D2H K
        e2e_sweeps += sum(info["iters"])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_vox = job_totals(e2e_s, float(e2e_sweeps * N3), world)
    h2d = sl.spheres.nbytes + N3
    d2h = N3 + 9 * 8

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        ctx.close()
        return

    # --- roofline of the dominant kernel -------------------------------------------
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    kinds = {k: v for k, v in trace.items() if v[1] > 0}
    total_ms = sum(v[0] for v in kinds.values())
    # the dominant kernel of the solve's own precision (FP64 correction passes are one kind)
    skip = ("other", "fp64") if args.precision == "fp32bulk" else ("other",)
    dom = max((k for k in kinds if k not in skip), key=lambda k: kinds[k][0])
    d_ms, d_n, d_bytes = kinds[dom]
    launch_s = d_ms / d_n / 1e3
    # algorithmic bytes per launch: 25 B (FP32) / 49 B (FP64) per voxel-iteration and
    # gradient -- read the field and the phase id, write the field -- times the voxels
    # of the three gradients one launch processes
    per_vox = 25.0 if prec == hmg.HMG_FP32_BULK else 49.0
    algo_bytes = per_vox * 3 * N3
    achieved = algo_bytes / launch_s / 1e9
    traffic, traffic_form = None, None
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            tinfo = json.load(fh)
        ent = tinfo.get(args.precision, {}).get(dom)
        if ent and ent.get("source_sha") == _kernel_sha():
            traffic = ent["dram_bytes_per_launch"]
            traffic_form = {"kernel": ent.get("form"), "algo_bytes_per_launch": ent.get("form_algo_bytes_per_launch")}
    except (OSError, ValueError):
        pass
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "algo_bytes_per_launch": algo_bytes, "algo_bytes_per_unit": per_vox,
                "units_per_launch": 3 * N3, "avg_launch_ms": d_ms / d_n,
                # the bytes this kernel's form moves (the x round trip also reads the
                # correction right-hand side or stores the field in some launches)
                "form_bytes_per_launch": d_bytes / d_n,
                "form_frac": (d_bytes / d_n) / launch_s / 1e9 / peak,
                "dram_frac": (traffic / launch_s / 1e9 / peak) if traffic else None,
                "traffic_form": traffic_form}
    kernels = {k: {"ms": v[0], "launches": v[1], "share": v[0] / total_ms,
                   "GBps": (v[2] / (v[0] / 1e3) / 1e9) if v[0] > 0 and v[2] > 0 else None}
               for k, v in kinds.items()}
    launches = int(sum(v[1] for v in kinds.values()))

    # accuracy of the timed solves: K against the oracle's stored result for this RVE
    # (FP64, written offline from the oracle alone) when there is one
    k_check = {}
    try:
        with open(os.path.join(ROOT, "tests", "golden", f"oracle_rsa{N_GRID}_s{seed}.json")) as fh:
            ref = json.load(fh)
        if ref["params"]["layer"] == LAYER and tuple(ref["params"]["k"]) == K_PHASES and ref["params"]["tol"] == TOL:
            Kref = np.array(ref["K"])
            k_check = {"k_err_vs_oracle": max(k_entry_err(Kk, Kref) for Kk in Ks),
                       "oracle_fp64_sweeps": int(sum(ref["iters"]))}
    except (OSError, ValueError, KeyError):
        pass

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == hmg.HMG_FP32_BULK else "f64", "data": "synthetic",
            "config": workload_config(args.precision),
            "solves_per_s": world * args.steps / (ms_max / 1e3),
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
            "sweeps_per_solve": sweeps / args.steps,
            "accuracy": {"k_err_definition": "max over entries of |K - Kref| / max(|Kref_ij|, 0.01 max_i Kref_ii)",
                         **k_check},
            "roofline": roofline,
            "algorithmic_hbm_frac": value / world * per_vox / (peak * 1e9),
            "kernels": kernels,
            "gpu_launches": launches * args.steps,
            "gpu_launches_note": "launches of one traced solve of the same RVE (outside the timed region) x steps",
            "z_variant": hmg.hmg_get_variant(ctx.handle, N_GRID),
            "clocks": clocks,
            "e2e": {"value": e2e_vox / e2e_s if e2e_vox else None, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}

    if not args.no_fp64 and prec == hmg.HMG_FP32_BULK:
        t = time.perf_counter()
        K64, info64, _ = hmg.hmg_solve(ctx.handle, phase_d, N_GRID, K_PHASES, TOL, hmg.HMG_FP64)
        dt = time.perf_counter() - t
        sw = sum(info64["iters"])
        rate = hmg.hmg_fp64_rate(ctx.handle)
        line["fp64_plain"] = {"voxel_iter_per_s": sw * N3 / dt, "solve_s": dt, "sweeps": sw,
                              "speedup_fp32bulk_solves": dt / (ms_max / 1e3 / args.steps),
                              "fp64_fma_rate_tflops": rate / 1e12}
        line["accuracy"]["k_err_vs_gpu_fp64"] = max(k_entry_err(Kk, K64) for Kk in Ks)
    # work-to-solution: voxel-iterations counted on the plain FP64 method's sweep count
    # (FP32 bulk runs more sweeps than FP64 to reach the same FP64 residuals)
    ref_sweeps = line["accuracy"].get("oracle_fp64_sweeps") or line.get("fp64_plain", {}).get("sweeps")
    if ref_sweeps:
        line["effective_voxel_iter_per_s"] = world * args.steps * ref_sweeps * N3 / (ms_max / 1e3)
        line["effective_note"] = "N^3 x (FP64 sweeps of the same RVE) per solve / solve time"
    if not args.no_cufft and prec == hmg.HMG_FP32_BULK:
        # comparison point: the same tau-form sweep on torch.fft (cuFFT) + torch pointwise ops
        sweep = torch_fft_sweep(phase_d, K_PHASES, N_GRID, "cuda")
        taus = [torch.ones((3, N_GRID, N_GRID, N_GRID), dtype=torch.float32, device="cuda") for _ in range(3)]
        grads = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
        reps = 8
        for j in range(3):
            taus[j] = sweep(taus[j], grads[j])
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(reps):
            for j in range(3):
                taus[j] = sweep(taus[j], grads[j])
        c1.record()
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        ours = ms / max(1, sweeps)
        line["cufft_comparison"] = {"voxel_iter_per_s": 3 * reps * N3 / (cms / 1e3),
                                    "ms_per_gradient_sweep": cms / (3 * reps),
                                    "ours_ms_per_gradient_sweep": ours,
                                    "ours_speedup": cms / (3 * reps) / ours,
                                    "note": "one tau-form sweep per gradient with torch.fft rfftn/irfftn (cuFFT) and "
                                            "torch pointwise ops, FP32, no residual, no defect correction; ours: the "
                                            "timed FP32-bulk solves (residuals, FP64 work included) per gradient sweep"}
        del taus
    if not args.no_cpu and world == 1:
        r = oracle_sample(oracle_phase(sl.spheres), 2)
        line["cpu_baseline"] = {"value": r["voxel_iters"] / r["seconds"], "unit": UNIT, "cores": r["threads"],
                                "kind": "oracle",
                                "sample": "2 oracle sweeps (steps 2-7, one gradient) of the 256^3 RVE, FP64"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


# ---------------------------------------------------------------------------
# many RVEs: batched solves and the request loop
# ---------------------------------------------------------------------------

def _spheres(args_tuple):
    from paper_1504_07499_gb300 import inputs as I
    seed, n, f = args_tuple
    return I.generate_spheres(seed, n, f).spheres


def _sphere_lists(specs):
    """Seeded sphere lists generated in parallel (spawned workers, before CUDA starts)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(specs), os.cpu_count() or 1)) as pool:
        return pool.map(_spheres, specs)


def run_batch(args) -> None:
    """Stochastic averaging batch: 64 RVEs (24 x 64^3, 24 x 96^3, 16 x 128^3), n ~ U{10..100},
    f ~ U[0.10, 0.40], l ~ U[0.1, 0.5], k 0.20/0.25/400, solved by hmg_solve_batch (every
    engine tick is one CUDA-graph launch over all RVEs); compared with the same RVEs solved
    one after the other (FP32 bulk) and with the plain FP64 method on a subset."""
    from paper_1504_07499_gb300 import inputs as I
    rec = I.batch_recipe()
    lists = _sphere_lists([(r["seed"], r["n"], r["f"]) for r in rec])
    import torch
    from paper_1504_07499_gb300 import build, hmg
    build.build()
    ctx = hmg.Context(0)
    phases, Ns = [], []
    for r, sph in zip(rec, lists):
        ph = torch.empty(r["N"] ** 3, dtype=torch.uint8, device="cuda")
        hmg.hmg_voxelize(ctx.handle, sph, r["layer"], r["N"], ph)
        phases.append(ph)
        Ns.append(r["N"])
    k3 = np.tile(np.array(K_PHASES), (len(rec), 1))
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        hmg.hmg_solve_batch(ctx.handle, phases, Ns, k3, TOL, hmg.HMG_FP32_BULK)
    t = time.perf_counter()
    vox = 0
    for _ in range(args.steps):
        K, infos, st = hmg.hmg_solve_batch(ctx.handle, phases, Ns, k3, TOL, hmg.HMG_FP32_BULK)
        vox += sum(N ** 3 * sum(i["iters"]) for N, i in zip(Ns, infos))
    dt = (time.perf_counter() - t) / args.steps
    # one after the other, same engine arithmetic per RVE
    t = time.perf_counter()
    vox_seq = 0
    for ph, N in zip(phases, Ns):
        _, info, _ = hmg.hmg_solve(ctx.handle, ph, N, K_PHASES, TOL, hmg.HMG_FP32_BULK)
        vox_seq += N ** 3 * sum(info["iters"])
    dt_seq = time.perf_counter() - t
    # plain FP64 on the first RVE of each size
    fp64 = {}
    for N in sorted(set(Ns)):
        i = Ns.index(N)
        t = time.perf_counter()
        _, info, _ = hmg.hmg_solve(ctx.handle, phases[i], N, K_PHASES, TOL, hmg.HMG_FP64)
        fp64[N] = {"solve_s": time.perf_counter() - t, "voxel_iter_per_s": N ** 3 * sum(info["iters"]) /
                   (time.perf_counter() - t)}
    est_fp64_s = sum(fp64[N]["solve_s"] for N in Ns)
    kbar = {}
    for N in sorted(set(Ns)):
        d = np.array([np.trace(K[i]) / 3 for i in range(len(Ns)) if Ns[i] == N])
        kbar[str(N)] = {"mean": float(d.mean()), "std": float(d.std(ddof=1)), "count": int(d.size)}
    line = {"metric": "voxel-iterations/s, 64 mixed-size RVEs in one engine (3 unit gradients, tol 1e-8)",
            "value": vox / args.steps / dt, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64: 24 x 64^3, 24 x 96^3, 16 x 128^3 RVEs (seeds 4000-4063), "
                                   "n ~ U{10..100}, f ~ U[0.10,0.40], l ~ U[0.1,0.5], k 0.20/0.25/400",
                       "precision": "fp32bulk", "total_voxels": int(sum(N ** 3 for N in Ns))},
            "solves_per_s": len(Ns) / dt,
            "sequential_fp32bulk": {"voxel_iter_per_s": vox_seq / dt_seq, "seconds": dt_seq,
                                    "batch_speedup": dt_seq / dt},
            "plain_fp64_estimate": {"seconds": est_fp64_s, "per_size": fp64, "batch_speedup": est_fp64_s / dt},
            "mean_K_trace_over_3": kbar,
            "status_all_ok": bool(st == hmg.HMG_OK)}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_contrast(args) -> None:
    """Contrast and layer sweep on the 256^3 RVE (100 spheres at 40 %, seed 3000): l in
    {0.1, 0.3, 0.5} x k_coat in {2, 40, 400, 4000} (contrast 10 .. 2e4 with k_min = 0.2),
    each solved in FP32 bulk and in plain FP64 to tol 1e-8.  Reports sweeps per gradient
    against the contraction bound ln(tol)/ln(rho), rho = (sqrt(c)-1)/(sqrt(c)+1), the
    throughput of both forms, the dominant FP32 kernel's bandwidth from the tracer and the
    two forms' K difference."""
    import torch
    from paper_1504_07499_gb300 import build, hmg
    from paper_1504_07499_gb300 import inputs as I
    build.build()
    ctx = hmg.Context(0)
    sl = I.generate_spheres(SEED, N_SPHERES, F_SP)
    sph_d = torch.from_numpy(np.ascontiguousarray(sl.spheres)).cuda()
    N = N_GRID
    peak = measured_peaks().get("hbm_gbs") or 6800.0
    ph = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    hmg.hmg_voxelize(ctx.handle, sph_d, 0.3, N, ph)
    hmg.hmg_solve(ctx.handle, ph, N, K_PHASES, TOL, hmg.HMG_FP32_BULK)     # autotune + warm-up
    cases, vox32, t32, vox64, t64 = [], 0.0, 0.0, 0.0, 0.0
    for layer in (0.1, 0.3, 0.5):
        hmg.hmg_voxelize(ctx.handle, sph_d, layer, N, ph)
        for kc in (2.0, 40.0, 400.0, 4000.0):
            k = (K_PHASES[0], K_PHASES[1], kc)
            c = max(k) / min(k)
            rho = (np.sqrt(c) - 1) / (np.sqrt(c) + 1)
            row = {"layer": layer, "k_coat": kc, "contrast": c, "bound_sweeps": float(np.log(TOL) / np.log(rho))}
            for name, prec in (("fp32bulk", hmg.HMG_FP32_BULK), ("fp64", hmg.HMG_FP64)):
                hmg.hmg_trace_enable(ctx.handle, True)
                torch.cuda.synchronize()
                t = time.perf_counter()
                K, info, st = hmg.hmg_solve(ctx.handle, ph, N, k, TOL, prec, allow=(hmg.HMG_OK, hmg.HMG_NOT_CONVERGED))
                dt = time.perf_counter() - t
                tr = hmg.hmg_trace_read(ctx.handle)
                hmg.hmg_trace_enable(ctx.handle, False)
                sweeps = int(sum(info["iters"]))
                ent = {"status": int(st), "sweeps_per_gradient": list(info["iters"]), "solve_s": dt,
                       "voxel_iter_per_s": N ** 3 * sweeps / dt, "K": K.tolist(),
                       "algorithmic_hbm_frac": N ** 3 * sweeps / dt * (25.0 if name == "fp32bulk" else 49.0) / 1e9 / peak}
                if name == "fp32bulk":
                    kinds = {kk: v for kk, v in tr.items() if v[1] > 0 and kk not in ("other", "fp64")}
                    dom = max(kinds, key=lambda kk: kinds[kk][0])
                    ms, n, b = kinds[dom]
                    ent["dominant_kernel"] = {"kind": dom, "GBps": b / (ms / 1e3) / 1e9, "frac": b / (ms / 1e3) / 1e9 / peak}
                    ent["fp64_rounds"] = int(info.get("fp64_rounds", 0))
                    vox32 += N ** 3 * sweeps
                    t32 += dt
                else:
                    vox64 += N ** 3 * sweeps
                    t64 += dt
                row[name] = ent
            K32, K64 = np.array(row["fp32bulk"]["K"]), np.array(row["fp64"]["K"])
            row["K_rel_diff"] = float(np.abs(K32 - K64).max() / np.abs(K64).max())
            cases.append(row)
            print(json.dumps({"case": row}), file=sys.stderr, flush=True)
    line = {"metric": "voxel-iterations/s at 256^3 over contrast 10..2e4 and layer 0.1..0.5 (3 unit gradients, tol 1e-8)",
            "value": vox32 / t32, "unit": UNIT, "n_gpus": 1, "steps": len(cases), "warmup": 1,
            "ms_per_step": 1e3 * t32 / len(cases), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "rsa256 contrast sweep: 256^3, 100 spheres at 40 % (seed 3000), l in {0.1,0.3,0.5}, "
                                   "k 0.20/0.25/{2,40,400,4000}", "precision": "fp32bulk"},
            "fp64_plain": {"voxel_iter_per_s": vox64 / t64, "seconds": t64, "speedup_fp32bulk": t64 / t32},
            "cases": cases}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_schemes(args) -> None:
    """The FFT-based schemes §3 lists, on the 256^3 RVE (100 spheres at 40 %, l = 0.3,
    seed 3000) at contrast 10, 200 and 2000 (k_coat 2, 40, 400), all in FP32 bulk to tol
    1e-8: accelerated (Eyre-Milton), augmented Lagrangian, the polarization iteration
    with relaxation 1.5, and the basic scheme; sweeps per gradient against each scheme's
    contraction bound, solve time, throughput, and the K difference to Eyre-Milton."""
    import torch
    from paper_1504_07499_gb300 import build, hmg
    from paper_1504_07499_gb300 import inputs as I
    build.build()
    ctx = hmg.Context(0)
    sl = I.generate_spheres(SEED, N_SPHERES, F_SP)
    N = N_GRID
    ph = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    hmg.hmg_voxelize(ctx.handle, torch.from_numpy(np.ascontiguousarray(sl.spheres)).cuda(), LAYER, N, ph)
    hmg.hmg_solve(ctx.handle, ph, N, K_PHASES, TOL, hmg.HMG_FP32_BULK)     # autotune + warm-up
    cases, vox, tt = [], 0.0, 0.0
    for kc in (2.0, 40.0, 400.0):
        k = (K_PHASES[0], K_PHASES[1], kc)
        c = max(k) / min(k)
        row = {"k_coat": kc, "contrast": c}
        rem = (np.sqrt(c) - 1) / (np.sqrt(c) + 1)
        for name, sch, rho in (("eyre_milton", hmg.HMG_SCHEME_EYRE_MILTON, rem),
                               ("augmented_lagrangian", hmg.HMG_SCHEME_AUGMENTED_LAGRANGIAN, 0.5 * (1 + rem)),
                               ("polarization_beta1.5", None, 1 - 0.75 * (1 - rem)),
                               ("basic", hmg.HMG_SCHEME_BASIC, (c - 1) / (c + 1))):
            torch.cuda.synchronize()
            t = time.perf_counter()
            if sch is None:
                K, info, st = hmg.hmg_solve_polarization(ctx.handle, ph, N, k, TOL, hmg.HMG_FP32_BULK, 1.5,
                                                         max_iter=200000, allow=(hmg.HMG_OK, hmg.HMG_NOT_CONVERGED))
            else:
                K, info, st = hmg.hmg_solve_scheme(ctx.handle, ph, N, k, TOL, hmg.HMG_FP32_BULK, sch,
                                                   max_iter=200000, allow=(hmg.HMG_OK, hmg.HMG_NOT_CONVERGED))
            dt = time.perf_counter() - t
            sweeps = int(sum(info["iters"]))
            row[name] = {"status": int(st), "sweeps_per_gradient": list(info["iters"]),
                         "bound_sweeps": float(np.log(TOL) / np.log(rho)), "solve_s": dt,
                         "voxel_iter_per_s": N ** 3 * sweeps / dt, "fp64_rounds": int(info.get("fp64_rounds", 0)),
                         "K": K.tolist()}
            vox += N ** 3 * sweeps
            tt += dt
        Ke = np.array(row["eyre_milton"]["K"])
        for name in ("augmented_lagrangian", "polarization_beta1.5", "basic"):
            row[name]["K_rel_diff_to_em"] = float(np.abs(np.array(row[name]["K"]) - Ke).max() / np.abs(Ke).max())
            row[name]["time_ratio_to_em"] = row[name]["solve_s"] / row["eyre_milton"]["solve_s"]
        cases.append(row)
        print(json.dumps({"case": row}), file=sys.stderr, flush=True)
    line = {"metric": "voxel-iterations/s at 256^3, four FFT-based schemes, contrast 10..2000 "
                      "(3 unit gradients, tol 1e-8)",
            "value": vox / tt, "unit": UNIT, "n_gpus": 1, "steps": 4 * len(cases), "warmup": 1,
            "ms_per_step": 1e3 * tt / (4 * len(cases)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "rsa256 scheme comparison: 256^3, 100 spheres at 40 % (seed 3000), l = 0.3, "
                                   "k 0.20/0.25/{2,40,400}", "precision": "fp32bulk"},
            "cases": cases}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_layers(args) -> None:
    """The paper's sweep over the coating layer (§5): phases matrix 1, inclusion 0.2, coating
    400 (contrast 2000), spheres at f_sp = 0.3 (coating included), n_sp in {30, 70, 100},
    l in {0.02, 0.04, 0.06, 0.08, 0.1, 0.2, ..., 0.9}, at 64^3, 128^3 (10 samples per point,
    seeds 6000 + s) and 256^3 (3 samples), FP32 bulk to tol 1e-8.  Reports the mean and
    standard deviation over samples of tr K / 3 (the paper's homogenized value), the largest
    off-diagonal / diagonal ratio, whether tr K / 3 never falls as l grows, for every sample (exact for
    the discrete problem: a thicker layer only raises voxel conductivities, from 0.2 to 400,
    and K is monotone in them), and whether the spread shrinks with the resolution."""
    import torch
    from paper_1504_07499_gb300 import build, hmg
    from paper_1504_07499_gb300 import inputs as I
    build.build()
    ctx = hmg.Context(0)
    k = (1.0, 0.2, 400.0)
    layers = (0.02, 0.04, 0.06, 0.08, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)
    plan = ((64, 10), (128, 10), (256, 3))
    lists = _sphere_lists([(6000 + smp, n, 0.3) for n in (30, 70, 100) for smp in range(10)])
    sph = {(n, smp): lists[i * 10 + smp] for i, n in enumerate((30, 70, 100)) for smp in range(10)}
    out, vox, tt, monotone, aniso = {}, 0.0, 0.0, True, 0.0
    for N, samples in plan:
        ph = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
        for n in (30, 70, 100):
            traces = np.zeros((samples, len(layers)))
            for smp in range(samples):
                sd = torch.from_numpy(np.ascontiguousarray(sph[(n, smp)])).cuda()
                for j, layer in enumerate(layers):
                    hmg.hmg_voxelize(ctx.handle, sd, layer, N, ph)
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    K, info, st = hmg.hmg_solve(ctx.handle, ph, N, k, TOL, hmg.HMG_FP32_BULK)
                    tt += time.perf_counter() - t
                    vox += N ** 3 * sum(info["iters"])
                    d = np.diag(K)
                    traces[smp, j] = d.mean()
                    aniso = max(aniso, float(np.abs(K - np.diag(d)).max() / d.mean()))
                # non-decreasing (equal where the voxelization does not change between two l)
                monotone &= bool((np.diff(traces[smp]) >= -1e-7 * traces[smp, 1:]).all())
            out[f"{N}/{n}"] = {"mean": traces.mean(0).tolist(), "std": traces.std(0, ddof=1).tolist(),
                               "samples": samples}
        print(json.dumps({"done": N}), file=sys.stderr, flush=True)
    shrink = [out[f"256/{n}"]["std"][j] < out[f"64/{n}"]["std"][j] for n in (30, 70, 100) for j in range(len(layers))]
    line = {"metric": "voxel-iterations/s over the paper's layer sweep (64^3, 128^3, 256^3; 3 unit gradients, tol 1e-8)",
            "value": vox / tt, "unit": UNIT, "n_gpus": 1, "steps": 3 * len(layers) * sum(s for _, s in plan),
            "warmup": 0, "ms_per_step": 1e3 * tt / (3 * len(layers) * sum(s for _, s in plan)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "paper layer sweep: k 1/0.2/400, f_sp 0.3, n_sp 30/70/100, l 0.02..0.9, "
                                   "10 samples at 64^3 and 128^3, 3 at 256^3 (seeds 6000+)", "precision": "fp32bulk",
                       "layers": list(layers)},
            "k_mean_over_samples": out, "rises_with_layer_every_sample": monotone,
            "max_offdiag_over_diag": aniso,
            "std_256_below_std_64_fraction": sum(shrink) / len(shrink)}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args) -> None:
    """Poisson stream of requests (seed 5000): N uniform over {64, 96, 128, 192, 256},
    k_coat over {40, 400, 4000}, 100 spheres at 40 %, l in {0.1, 0.3, 0.5}, FP32 bulk,
    through hmg_submit / hmg_poll at 0.5x, 1x and 1.5x the rate sequential FP32-bulk
    solves sustain.  Sequential FP32-bulk and plain-FP64 service of the same arrivals is
    simulated from measured per-request service times (FIFO, one at a time)."""
    from paper_1504_07499_gb300 import inputs as I
    pool_specs = [(5000 + i, 100, 0.40) for i in range(4)]
    lists = _sphere_lists(pool_specs)
    import torch
    from paper_1504_07499_gb300 import build, hmg
    build.build()
    u = I.SplitMix64(5000, 17).uniform(4 * args.requests).reshape(args.requests, 4)
    sizes, kcs, layers = (64, 96, 128, 192, 256), (40.0, 400.0, 4000.0), (0.1, 0.3, 0.5)
    reqs = [(sizes[int(a * 5)], kcs[int(b * 3)], layers[int(c * 3)], int(d * 4)) for a, b, c, d in u]
    ctx = hmg.Context(0)
    phase_cache = {}
    for N, kc, layer, li in reqs:
        key = (N, layer, li)
        if key not in phase_cache:
            ph = np.empty(N ** 3, dtype=np.uint8)
            hmg.hmg_voxelize(ctx.handle, lists[li], layer, N, ph)
            phase_cache[key] = ph
    # service times of sequential solves (FP32 bulk; plain FP64 per (N, k_coat) class)
    svc32, svc64 = [], {}
    for N, kc, layer, li in reqs:
        t = time.perf_counter()
        hmg.hmg_solve(ctx.handle, phase_cache[(N, layer, li)], N, (0.20, 0.25, kc), TOL, hmg.HMG_FP32_BULK)
        svc32.append(time.perf_counter() - t)
    for N, kc, layer, li in reqs:
        if (N, kc) not in svc64 and N <= 128:
            t = time.perf_counter()
            hmg.hmg_solve(ctx.handle, phase_cache[(N, layer, li)], N, (0.20, 0.25, kc), TOL, hmg.HMG_FP64)
            svc64[(N, kc)] = time.perf_counter() - t
    ctx.close()
    # larger classes: scale the measured FP64 time of the same contrast by the voxel count
    def fp64_time(N, kc):
        if (N, kc) in svc64:
            return svc64[(N, kc)]
        base = max((n for (n, k) in svc64 if k == kc), default=None)
        return svc64[(base, kc)] * (N / base) ** 3 * np.log2(N) / np.log2(base)

    def fifo(arrivals, service):
        done, lat = 0.0, []
        for a, s in zip(arrivals, service):
            done = max(done, a) + s
            lat.append(done - a)
        return done, lat

    mean32 = float(np.mean(svc32))
    results = []
    for factor in (0.5, 1.0, 1.5):
        rate = factor / mean32
        arr = I.poisson_arrivals(5000, rate, len(reqs))
        c = hmg.Context(0)
        tickets, t0 = [], time.perf_counter()
        for (N, kc, layer, li), a in zip(reqs, arr):
            while time.perf_counter() - t0 < a:
                time.sleep(0.0005)
            tickets.append(hmg.hmg_submit(c.handle, phase_cache[(N, layer, li)], N, (0.20, 0.25, kc), TOL,
                                          hmg.HMG_FP32_BULK))
        lat, pending = [], set(tickets)
        while pending:
            for t in list(pending):
                st, K, info = hmg.hmg_poll(c.handle, t)
                if st != hmg.HMG_PENDING:
                    lat.append(info["seconds"])
                    pending.discard(t)
            time.sleep(0.002)
        makespan = time.perf_counter() - t0
        stats = hmg.hmg_server_stats(c.handle)
        c.close()
        end32, lat32 = fifo(arr, svc32)
        end64, lat64 = fifo(arr, [fp64_time(N, kc) for N, kc, _, _ in reqs])
        results.append({"rate_factor": factor, "rate_hz": rate, "solves_per_s": len(reqs) / makespan,
                        "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                        "max_resident": stats["max_resident"], "graph_launches": stats["graph_launches"],
                        "sequential_fp32bulk": {"solves_per_s": len(reqs) / end32,
                                                "p50_ms": 1e3 * float(np.percentile(lat32, 50)),
                                                "p99_ms": 1e3 * float(np.percentile(lat32, 99))},
                        "sequential_fp64": {"solves_per_s": len(reqs) / end64,
                                            "p50_ms": 1e3 * float(np.percentile(lat64, 50)),
                                            "p99_ms": 1e3 * float(np.percentile(lat64, 99))}})
    line = {"metric": "solves/s and p50/p99 latency of a Poisson request stream (serving)",
            "value": results[-1]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": len(reqs),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serve: N in {64,96,128,192,256}, k_coat in {40,400,4000}, 100 spheres at 40%, "
                                   "l in {0.1,0.3,0.5}, Poisson arrivals seed 5000", "requests": len(reqs),
                       "mean_sequential_fp32bulk_service_s": mean32,
                       "fp64_service_measured": {f"{k[0]}/{k[1]}": v for k, v in svc64.items()}},
            "rates": results}
    print(json.dumps(line), flush=True)


# the sources of the sweep kernels (device code and the headers it includes); host-side
# driver, engine and request-loop files do not change what a kernel moves
KERNEL_SOURCES = ("hmg_fast.cu", "hmg_kernels.cu", "hmg_fused.cu", "hmg_internal.h")


def _kernel_sha() -> str:
    """Hash of the sweep kernels' code (comments and blank lines left out), which ties a
    stored ncu measurement to the code it was taken on."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1504_07499_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in KERNEL_SOURCES or f.endswith(".cuh"):
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
            for line in text.splitlines():
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
