#!/usr/bin/env python3
"""Benchmark: aligned curve pairs/s at N = 1024 on one GB300 (per rank).

Workload (one "step"): 4096 curve pairs given as raw, non-uniformly sampled
point lists (N_in ~ U{500..2000} nodes per curve, node parameters jittered by
+-40% of the mean spacing, Fourier-series shapes with up to 16 harmonics);
both curves of every pair are resampled on the GPU to N = 1024 nodes uniform
in arc length (fa_resample_arclength), then every pair is aligned over all
cyclic shifts and rotations with the FFT method (fa_align_pairs, FA_FFT),
all in FP64.  Inputs are resident in HBM when the timed region starts; the
raw nodes (~164 MB) exceed the 129 MB L2, so no extra flush is needed.

The JSON line also carries: the direct O(N^2) GPU baseline on the same
curves, the roofline of the dominant kernel (FP64 pipe: algorithmic FP64
flops per launch / CUDA-event time, against this GPU's FP64 FMA peak measured
in the same run), the end-to-end number through fa_align_curves_host with
pinned host buffers (copies inside the timed region), SM clocks sampled during
the timed region, and the CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle (the plain O(N^2) Kabsch search plus the
periodic-spline resampling, FP64, OpenMP over pairs) on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

P_PAIRS = 4096
N_NODES = 1024
N_MIN, N_MAX = 500, 2000
SEED = 1002
# DRAM bytes per launch of the bench workload's kernels come from one ncu capture
# each, recorded in profiles/dram_traffic.txt with a hash of the kernel's sources
# at capture time; a kernel whose sources have changed since reports no traffic.
TRAFFIC_FILE = Path(__file__).resolve().parent / "profiles" / "dram_traffic.txt"
KERNEL_SOURCES = {
    "resample_kernel": ("resample.cu", "df.cuh"),
    "align_fft_kernel": ("align_fft.cu", "fft_stages.cuh", "align_common.cuh"),
}


def kernel_source_hash(kernel: str) -> str:
    """First 16 hex digits of the SHA-256 of the kernel's source files."""
    csrc = Path(__file__).resolve().parent / "paper_2501_17779_gb300" / "csrc"
    hsh = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        hsh.update((csrc / name).read_bytes())
    return hsh.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """(bytes per launch, note) from the traffic file, or (None, why not)."""
    if kernel not in KERNEL_SOURCES or not TRAFFIC_FILE.exists():
        return None, "no capture recorded for this kernel"
    want = kernel_source_hash(kernel)
    for line in TRAFFIC_FILE.read_text().splitlines():
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel:
            if f[1] != want:
                return None, f"capture is of kernel sources {f[1]}, current {want}: stale"
            return float(f[2]) + float(f[3]), f"ncu capture of kernel sources {want}"
    return None, "no capture recorded for this kernel"
METRIC = "aligned curve pairs/s at N=1024 (FFT vs direct O(N²), 1 GB300); roofline fraction"
WORKLOAD = ("4096 pairs of raw curves (N_in ~ U{500..2000}, +-40% node jitter, <=16 harmonics), "
            "GPU arc-length resampling to N=1024 + FFT alignment over all shifts, FP64")
FP64_NOMINAL_TFLOPS = 1.25


# ----------------------------------------------------- algorithmic counts ---
def measured_hbm_gbs():
    """HBM copy bandwidth (GB/s) measured on this GPU type, from the peaks file
    at the repository root, or None when it is absent."""
    f = Path(__file__).resolve().parent / "MEASURED_PEAKS.json"
    try:
        return float(json.loads(f.read_text())["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def fft_flops(logn: int) -> int:
    """FP64 flops (FMA = 2) of one forward transform in the kernel's algorithm:
    an optional radix-2 stage (4 real adds per butterfly), then radix-4
    Stockham stages: 16 adds per butterfly in an untwiddled stage, four FMA-form
    butterflies (24 DFMA = 48 flops) per twiddled radix-4 butterfly."""
    N = 1 << logn
    q = N // 4
    fl = 0
    stages4 = logn // 2
    first_twiddled = False
    if logn & 1:
        fl += (N // 2) * 4
        first_twiddled = True
    for i in range(stages4):
        fl += q * (48 if (i > 0 or first_twiddled) else 16)
    return fl


def align_fft_flops_per_pair(logn: int) -> int:
    N = 1 << logn
    # 3 transforms; spectrum product 6/bin; |c|^2 3/shift; c(s*) 8/node; energy 12/node
    return 3 * fft_flops(logn) + 6 * N + 3 * N + 8 * N + 12 * N


def resample_flops(n_in: np.ndarray, N: int) -> int:
    """FP64 flops of fa_resample_arclength, counted from the kernel's algorithm
    (FMA = 2; a reciprocal, reciprocal square root or square root = 1):
      per input node: chord vector 2, |.|^2 3, rsqrt 1, length 1, chunk sum 1 = 8
      per interior node (n - P of them, P chunks): arc length 1, unit direction
        2, right-hand side 2, diagonal 2, pivot 2 + reciprocal 1, c' 1, y' 6,
        g' 2 (forward sweep 19); first-interior recurrence 7; M sweep 8 = 34
      per chunk: interface row 6, reduced row 14, 18 per cyclic-reduction
        level (log2 P - 1 levels), final 2x2 solve 14, minus the recurrence's
        missing last step 7
      per output node: parameter 1, local coordinate 2, cubic weights 8,
        spline value 12, mean sum 2, perimeter chord 7, centring and scaling 4 = 36
      per curve: warp scans and reductions 640, scalars 10."""
    n = np.asarray(n_in, np.int64)
    P = np.full(n.shape, 32, np.int64)
    for _ in range(5):
        P = np.where(2 * P > n, P // 2, P)
    levels = np.log2(np.maximum(P, 1)).astype(np.int64) - 1
    per_chunk = 6 + 14 + 18 * levels + 14 - 7
    tot = 8 * n + 34 * (n - P) + per_chunk * P + 36 * N + 650
    return int(tot.sum())


def elastic_flops(lm_steps: np.ndarray, iters: np.ndarray, N: int) -> int:
    """FP64 flops (FMA = 2) of fa_elastic_distance, counted from the kernel's
    algorithm per unit of work (the float32 lattice programme is not FP64
    work and is left out):
      per refinement (Levenberg-Marquardt) step and node: the trial point's
        cell pass 180 (Catmull-Rom value, slope and curvature of q2 at the
        cell midpoint 96, sqrt of the slope 2, residual 10, Jacobian and
        curvature terms 52, reductions 20), the normal-equation rows 40, the
        three-right-hand-side tridiagonal solve counted as Thomas 18, the
        Schur-complement sums 10, the step and its shortening 12 = 260
      per outer iteration ((t0,R)-step): two transforms 10 N log2 N, the
        reparameterised samples 36 N, product, |c|^2, c(s*), energy 27 N
      per pair: the pre-alignment (three transforms 15 N log2 N, product,
        |c|^2 and c(s*) 17 N), the SRV samples of both curves 24 N, the
        arc-length resampling of both curves 2 (42 + 36) N"""
    lg = int(np.log2(N))
    steps = np.asarray(lm_steps, np.int64).sum()
    it = np.asarray(iters, np.int64).sum()
    P = np.asarray(iters).size
    return int(260 * N * steps + (10 * N * lg + 63 * N) * it + P * (15 * N * lg + 197 * N))


def ragged_flops(sizes: np.ndarray) -> int:
    """FP64 flops of fa_align_pairs_ragged: per pair with transform length L =
    R B (B <= 4096): 3R transforms of length B, the spectrum product (6 per
    bin), the radix-R input stage and output recombination (complex products
    for R > 1), |c|^2, c(s*) and the energy over the n nodes."""
    tot = 0
    for n in np.asarray(sizes, np.int64):
        n = int(n)
        L = n if n & (n - 1) == 0 else 1 << (2 * n - 1).bit_length()
        B = min(L, 4096)
        R = L // B
        logb = B.bit_length() - 1
        tot += 3 * R * fft_flops(logb) + 6 * L
        if R > 1:
            tot += 2 * (R - 1) * B * 6 + (R - 1) * 8 * n
        tot += 3 * n + 8 * n + 12 * n
    return tot


def direct_flops_per_pair(N: int) -> int:
    return 8 * N * N + 3 * N + 12 * N


# ------------------------------------------------------------- clocks ------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- helpers ----
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, pg=None, device=None) -> float:
    """The slowest rank's time, known to every rank (an all-reduce MAX over
    the process group; the identity for one process)."""
    if pg is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, steps: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed in `steps` steps
    over the slowest rank's time `ms` (milliseconds)."""
    return world * units_per_rank * steps / (ms * 1e-3)


def make_workload(rank: int, P: int = P_PAIRS):
    from paper_2501_17779_gb300 import synth

    return synth.raw_pairs(SEED + 1000 * rank, P=P, n_min=N_MIN, n_max=N_MAX)


def oracle_sample(rp, n_pairs: int, N: int, nthreads: int):
    """Run the oracle (resampling + exhaustive alignment) on the first
    n_pairs pairs of a workload; returns seconds of wall time and the
    result (with the oracle's resampled curves under "z1", "z2")."""
    import oracle

    P = rp.offsets.size // 2
    idx = list(range(n_pairs)) + list(range(P, P + n_pairs))
    curves = [rp.pts[rp.offsets[i]:rp.offsets[i + 1]] for i in idx]
    offs = np.concatenate([[0], np.cumsum([c.size for c in curves])]).astype(np.int64)
    pts = np.concatenate(curves)
    t0 = time.perf_counter()
    z, st = oracle.resample(pts, offs, N, nthreads=nthreads)
    res = oracle.align_pairs(z[:n_pairs], z[n_pairs:], nthreads=nthreads)
    secs = time.perf_counter() - t0
    res["z1"], res["z2"] = z[:n_pairs], z[n_pairs:]
    return secs, res


# Parity bounds of the bench's own comparison (the oracle resamples the raw
# curves itself).  Resampled nodes agree to NODE_TOL; on equal inputs the FP64
# aligner agrees to 1e-12 relative energy and 1e-10 rad.  Perturbing every node
# by at most dz moves the optimal energy E = h sum |z1 - R z2|^2 by at most
# 2 sqrt(E) (2 dz) + (2 dz)^2, and h c(s*) by at most dz (sqrt(n1) + sqrt(n2)),
# n_i = h sum |z_i|^2 (Cauchy-Schwarz), so theta = arg c by that over h|c| =
# (n1 + n2 - E) / 2.  complex64 storage rounds every node by at most
# 2^-24 max|z| per coordinate; a pair whose shift differs from the oracle's is
# a tie when the two energies differ by no more than that perturbation allows.
NODE_TOL = 1e-12


def parity_vs_oracle(o, shift, theta, energy, zmax=None) -> dict:
    """GPU results of the first pairs against the oracle's, with the per-pair
    bounds above: FP64 paths (zmax None) with node agreement NODE_TOL and
    FP64 aligner tolerances; complex64 storage (zmax = the largest |z| of the
    resampled curves, which sizes the rounding) with |dtheta| <= 1e-5 and
    relative dE <= 1e-5 where the shifts agree, ties counted as agreement."""
    n = o["shift"].size
    s = shift[:n].cpu().numpy()
    th = theta[:n].cpu().numpy()
    e = energy[:n].cpu().numpy()
    z1, z2 = o["z1"], o["z2"]
    h = 1.0 / z1.shape[1]
    n1 = h * (np.abs(z1) ** 2).sum(1)
    n2 = h * (np.abs(z2) ** 2).sum(1)
    E = np.maximum(o["energy"], 0.0)
    if zmax is None:
        dz, e_rel, th_tol, kind = NODE_TOL, 1e-12, 1e-10, "fp64"
    else:
        dz, e_rel, th_tol, kind = NODE_TOL + 2.0 ** -24 * np.sqrt(2.0) * zmax, 1e-5, 1e-5, "c64"
    e_move = 2.0 * np.sqrt(E) * (2 * dz) + (2 * dz) ** 2
    e_tol = e_rel * E + (e_move if kind == "fp64" else 0.0)
    th_bound = th_tol + (dz * (np.sqrt(n1) + np.sqrt(n2)) / np.maximum((n1 + n2 - E) / 2, 1e-300)
                         if kind == "fp64" else 0.0)
    same = s == o["shift"]
    de = np.abs(e - o["energy"])
    # a different shift: a tie of the oracle's energies (the parity rule, 1e-9)
    # or, for complex64 storage, within the energy change its rounding allows
    tie = ~same & (de <= (1e-9 if kind == "fp64" else 2 * e_move + 1e-9))
    dth = np.abs(np.angle(np.exp(1j * (th - o["theta"]))))
    agree_tie = float((same | tie).mean())
    ok_th = bool((dth[same] <= th_bound if np.ndim(th_bound) == 0 else
                  dth[same] <= th_bound[same]).all())
    ok_e = bool((de[same] <= e_tol[same]).all())
    need = 1.0 if kind == "fp64" else 0.999
    return {"pairs": int(n), "shift_agreement": float(same.mean()),
            "shift_agreement_or_tie": agree_tie,
            "max_abs_dtheta": float(dth[same].max()) if same.any() else None,
            "max_rel_denergy": float((de / o["energy"]).max()),
            "max_denergy_over_bound": float((de[same] / e_tol[same]).max()) if same.any() else None,
            "bound": ("energy: 1e-12 E + 2 sqrt(E) 2dz + (2dz)^2 with dz = 1e-12 (nodes); "
                      "theta: 1e-10 + dz (sqrt(n1) + sqrt(n2)) / h|c|; shifts: exact or a "
                      "1e-9 tie, on every pair" if kind == "fp64" else
                      "relative energy 1e-5 and theta 1e-5 where the shift agrees; shift "
                      "agreement >= 0.999 counting ties within the energy change complex64 "
                      "rounding allows (dz = 2^-24 sqrt(2) max|z|)"),
            "within_bound": bool(ok_th and ok_e and agree_tie >= need)}


# ------------------------------------------------------------ reference ----
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    nthreads = os.cpu_count() or 1
    rp = make_workload(0, P=max(args.ref_pairs, 8))
    for _ in range(args.warmup):
        oracle_sample(rp, min(8, args.ref_pairs), N_NODES, nthreads)
    times = [oracle_sample(rp, args.ref_pairs, N_NODES, nthreads)[0] for _ in range(args.steps)]
    tot = sum(times)
    value = args.ref_pairs * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs": P_PAIRS, "N": N_NODES,
                   "sample_pairs_per_step": args.ref_pairs},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"{args.ref_pairs} pairs of the 4096-pair workload per step "
                                   "(resampling + O(N^2) Kabsch search)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU ------
def run_gpu(args):
    import torch

    from paper_2501_17779_gb300 import _lib, api, build as pbuild

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    pbuild.build()
    L = _lib.load()
    h = api.handle(local)

    rp = make_workload(rank)
    P, N = P_PAIRS, N_NODES
    C = 2 * P
    n_in = np.diff(rp.offsets)
    pts = torch.from_numpy(rp.pts).to(dev)
    offs = torch.from_numpy(rp.offsets).to(dev)
    n_pts = pts.numel()
    z = torch.empty((C, N), dtype=torch.complex128, device=dev)
    rst = torch.empty(C, dtype=torch.int8, device=dev)
    ws_bytes = int(L.fa_resample_workspace_size(C, n_pts, N, _lib.CENTER | _lib.UNIT_LENGTH))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    shift = torch.empty(P, dtype=torch.int32, device=dev)
    theta = torch.empty(P, dtype=torch.float64, device=dev)
    energy = torch.empty(P, dtype=torch.float64, device=dev)
    ast = torch.empty(P, dtype=torch.int8, device=dev)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    z1p = z.data_ptr()
    z2p = z1p + P * N * 16
    flags = _lib.CENTER | _lib.UNIT_LENGTH

    def resample():
        _lib.check(L.fa_resample_arclength(h, pts.data_ptr(), offs.data_ptr(), C, n_pts, N, flags,
                                           z.data_ptr(), rst.data_ptr(), ws.data_ptr(), ws_bytes,
                                           sptr))

    def align(method=_lib.FFT, prec=_lib.PREC_FP64):
        _lib.check(L.fa_align_pairs(h, z1p, z2p, P, N, _lib.Z_F64, method, prec,
                                    shift.data_ptr(), theta.data_ptr(), energy.data_ptr(),
                                    ast.data_ptr(), sptr))

    def barrier():
        torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (also validates statuses once)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            resample()
            align()
    torch.cuda.synchronize(dev)
    assert int((rst != 0).sum()) == 0 and int((ast != 0).sum()) == 0, "bad status in workload"

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            t_start.record(stream)
            for k in range(K):
                ev[k][0].record(stream)
                resample()
                ev[k][1].record(stream)
                align()
                ev[k][2].record(stream)
            t_end.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    total_ms = t_start.elapsed_time(t_end)
    rs_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    al_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    total_ms = max_over_ranks(total_ms, pg, dev)
    value = job_rate(world, P, K, total_ms)

    # direct O(N^2) baseline on the same resampled curves (align step only)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        align(_lib.DIRECT)
        e0.record(stream)
        reps = max(1, args.direct_reps)
        for _ in range(reps):
            align(_lib.DIRECT)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    direct_ms = e0.elapsed_time(e1) / reps

    # FA_PREC_MIXED variant of the alignment step on the same curves (the three
    # transforms in double-float, c(s*), theta and the energy in FP64); also
    # checks it picks the FP64 search's shifts
    with torch.cuda.stream(stream):
        align()
        ref_shift = shift.clone()
        ref_energy = energy.clone()
        align(prec=_lib.PREC_MIXED)
        e0.record(stream)
        for _ in range(K):
            align(prec=_lib.PREC_MIXED)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    mixed_ms = e0.elapsed_time(e1) / K
    mix_res = (shift.clone(), theta.clone(), energy.clone())
    same = shift == ref_shift
    mixed_agree = float(same.double().mean().item())
    mixed_tie_ok = bool(((energy - ref_energy).abs()[~same] <= 1e-9).all().item())
    ref_theta = None
    with torch.cuda.stream(stream):
        align()
        ref_theta = theta.clone()
    torch.cuda.synchronize(dev)

    # FP32-storage variant of the whole step: resampled nodes stored as
    # complex64 (FA_STORE_FP32), aligned in FP64 from them (FA_Z_F32); errors
    # against the FP64-storage results of the same curves
    zmax = float(z.abs().max().item())
    z32 = torch.empty((C, N), dtype=torch.complex64, device=dev)
    ws32_bytes = int(L.fa_resample_workspace_size(C, n_pts, N, flags | _lib.STORE_FP32))
    ws32 = torch.empty(ws32_bytes, dtype=torch.uint8, device=dev)
    sh32 = torch.empty(P, dtype=torch.int32, device=dev)
    th32 = torch.empty(P, dtype=torch.float64, device=dev)
    en32 = torch.empty(P, dtype=torch.float64, device=dev)
    st32 = torch.empty(P, dtype=torch.int8, device=dev)

    def resample32():
        _lib.check(L.fa_resample_arclength(h, pts.data_ptr(), offs.data_ptr(), C, n_pts, N,
                                           flags | _lib.STORE_FP32, z32.data_ptr(), rst.data_ptr(),
                                           ws32.data_ptr(), ws32_bytes, sptr))

    def align32():
        _lib.check(L.fa_align_pairs(h, z32.data_ptr(), z32.data_ptr() + P * N * 8, P, N,
                                    _lib.Z_F32, _lib.FFT, _lib.PREC_FP64, sh32.data_ptr(),
                                    th32.data_ptr(), en32.data_ptr(), st32.data_ptr(), sptr))

    ev32 = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    with torch.cuda.stream(stream):
        resample32()
        align32()
        e0.record(stream)
        for k in range(K):
            ev32[k][0].record(stream)
            resample32()
            ev32[k][1].record(stream)
            align32()
            ev32[k][2].record(stream)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    f32_ms = e0.elapsed_time(e1) / K
    rs32_ms = statistics.mean(ev32[k][0].elapsed_time(ev32[k][1]) for k in range(K))
    al32_ms = statistics.mean(ev32[k][1].elapsed_time(ev32[k][2]) for k in range(K))
    same32 = sh32 == ref_shift
    dth32 = torch.remainder(th32 - ref_theta + np.pi, 2 * np.pi) - np.pi
    dz32 = 2.0 ** -24 * np.sqrt(2.0) * zmax
    move32 = 2.0 * torch.sqrt(ref_energy.clamp(min=0)) * (2 * dz32) + (2 * dz32) ** 2
    tie32 = ~same32 & ((en32 - ref_energy).abs() <= 2 * move32 + 1e-9)
    fp32_storage = {
        "ms_per_step": f32_ms, "pairs_per_s": world * P / (f32_ms * 1e-3),
        "shift_agreement_with_fp64": float(same32.double().mean().item()),
        "shift_agreement_with_fp64_or_tie": float((same32 | tie32).double().mean().item()),
        "tie": "a different shift whose energy is within 2 (2 sqrt(E) 2dz + (2dz)^2) + 1e-9 "
               "of the FP64 path's, dz = 2^-24 sqrt(2) max|z| (complex64 rounding of the nodes)",
        "max_abs_dtheta_where_shift_agrees": float(dth32.abs()[same32].max().item()),
        "max_rel_denergy": float(((en32 - ref_energy).abs() / ref_energy.abs()).max().item()),
        "dtype": "f64 compute, complex64 resampled nodes",
        "kernels_ms": {"resample_kernel<fp32 store>": rs32_ms, "align_fft_kernel<float2>": al32_ms}}
    del z32, ws32

    # FP64 peak measured in this run (denominator of the roofline)
    peak_lib = ctypes.CDLL(str(pbuild.build_probe()))
    peak_lib.fa_probe_fp64_fma_tflops.restype = ctypes.c_double
    peak_lib.fa_probe_fp64_fma_tflops.argtypes = [ctypes.c_int]
    fp64_peak = float(peak_lib.fa_probe_fp64_fma_tflops(5))

    # roofline of the dominant kernel
    rs_avg = statistics.mean(rs_ms)
    al_avg = statistics.mean(al_ms)
    fl_rs = resample_flops(n_in, N)
    fl_al = align_fft_flops_per_pair(10) * P
    kernels = {
        "resample_kernel": {"ms": rs_avg, "tflops": fl_rs / (rs_avg * 1e-3) / 1e12,
                            "flops_per_launch": fl_rs},
        "align_fft_kernel": {"ms": al_avg, "tflops": fl_al / (al_avg * 1e-3) / 1e12,
                             "flops_per_launch": fl_al},
    }
    for kv in kernels.values():  # each kernel against the same measured FP64 peak
        kv["frac_of_measured_fp64_peak"] = kv["tflops"] / fp64_peak
    # the FP32-storage variant against both rooflines: its arithmetic is the
    # same FP64 work, its algorithmic HBM bytes are 16 B per raw node read + 8 B
    # per resampled node written (resampling) and 8 B per node of both curves
    # read (alignment); the binding one is the larger fraction
    hbm_peak = measured_hbm_gbs()
    bytes_rs32 = 16 * int(n_pts) + 8 * C * N + 8 * (C + 1)
    bytes_al32 = 2 * P * N * 8 + 21 * P
    roof32 = {}
    for name, fl, by, ms in (("resample_kernel<fp32 store>", fl_rs, bytes_rs32, rs32_ms),
                             ("align_fft_kernel<float2>", fl_al, bytes_al32, al32_ms)):
        f_fp64 = fl / (ms * 1e-3) / 1e12 / fp64_peak
        f_hbm = (by / (ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None
        roof32[name] = {"ms": ms, "flops_per_launch": fl, "bytes_per_launch": by,
                        "frac_of_measured_fp64_peak": f_fp64, "frac_of_measured_hbm": f_hbm,
                        "bound": "alu" if f_hbm is None or f_fp64 >= f_hbm else "hbm"}
    fp32_storage["roofline"] = {"kernels": roof32, "fp64_peak_tflops": fp64_peak,
                                "hbm_peak_gbs": hbm_peak, "of": "measured",
                                "note": "no FP32-pipe roofline: the variant computes in FP64"}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    if args.traffic is not None:
        traffic, tnote = args.traffic, "given on the command line"
    else:
        traffic, tnote = recorded_traffic(dom)
    roof = {"bound": "alu", "kernel": dom, "achieved": kernels[dom]["tflops"], "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": kernels[dom]["tflops"] / fp64_peak,
            "traffic": traffic, "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum "
            f"per launch: {tnote}",
            "peak_kind": "FP64 FMA throughput measured in this run "
            f"(nominal {FP64_NOMINAL_TFLOPS})", "of": "measured"}

    # end to end through the C ABI with pinned host buffers
    pts_h = torch.from_numpy(rp.pts).pin_memory()
    offs_h = torch.from_numpy(rp.offsets).pin_memory()
    outs_h = (torch.empty(P, dtype=torch.int32).pin_memory(),
              torch.empty(P, dtype=torch.float64).pin_memory(),
              torch.empty(P, dtype=torch.float64).pin_memory(),
              torch.empty(P, dtype=torch.int8).pin_memory())
    with torch.cuda.stream(stream):
        for _ in range(2):
            api.align_curves_host(pts_h, offs_h, N, out=outs_h, device=local)
        barrier()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            api.align_curves_host(pts_h, offs_h, N, out=outs_h, device=local)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, pg, dev)

    # all-pairs alignment matrix: M = 2048 curves at N = 512 (fa_align_all_pairs)
    allp = None
    if not args.no_all_pairs:
        from paper_2501_17779_gb300 import synth

        Ma, Na = 2048, 512
        ap = synth.aligned_pairs(SEED + 7, P=Ma // 2, N=Na, n_harm=12, oversample=16)
        za = torch.from_numpy(np.concatenate([ap.z1, ap.z2])).to(dev)
        with torch.cuda.stream(stream):
            api.align_all_pairs(za)  # warm-up (allocates outputs and workspace)
            outs = api.align_all_pairs(za)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            reps = 3
            for _ in range(reps):
                api.align_all_pairs(za)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        all_ms = e0.elapsed_time(e1) / reps
        with torch.cuda.stream(stream):
            mouts = api.align_all_pairs(za, prec="mixed")
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(reps):
                api.align_all_pairs(za, prec="mixed")
            e1.record(stream)
        torch.cuda.synchronize(dev)
        all_mixed_ms = e0.elapsed_time(e1) / reps
        same = mouts[0] == outs[0]
        all_mixed_agree = float(same.double().mean().item())
        all_mixed_tie_ok = bool(((mouts[2] - outs[2]).abs()[~same] <= 1e-9).all().item())
        npairs = Ma * (Ma - 1) // 2
        fl_all = npairs * (fft_flops(9) + 29 * Na) + Ma * fft_flops(9)
        allp = {"workload": "2048 curves, N=512, every ordered pair (FP64)",
                "ms": all_ms, "ordered_pairs_per_s": Ma * (Ma - 1) / (all_ms * 1e-3),
                "searched_pairs": npairs, "tflops": fl_all / (all_ms * 1e-3) / 1e12,
                "frac_of_fp64_peak": fl_all / (all_ms * 1e-3) / 1e12 / fp64_peak,
                "status_ok": bool((outs[3] == 0).all().item()),
                "mixed": {"ms": all_mixed_ms, "ordered_pairs_per_s": Ma * (Ma - 1) / (all_mixed_ms * 1e-3),
                          "speedup_vs_fp64": all_ms / all_mixed_ms,
                          "shift_agreement_with_fp64": all_mixed_agree,
                          "disagreements_within_tie": all_mixed_tie_ok,
                          "dtype": "double-float (f32x2) search + f64 c(s*)/theta/energy"}}
        # tensor-core search (DFT of the cross-spectra as a tcgen05 GEMM, top 8
        # shifts per pair re-scored in double-float) on the matrix stored as
        # complex64, against the FP64 search of the same complex64 input
        z32 = za.to(torch.complex64)
        with torch.cuda.stream(stream):
            ref32 = api.align_all_pairs(z32)
        torch.cuda.synchronize(dev)
        tc = {}
        for prec, terms in (("tc_bf16x3", 3), ("tc_fp16x3", 3), ("tc_tf32x3", 3), ("tc_tf32", 1)):
            with torch.cuda.stream(stream):
                touts = api.align_all_pairs(z32, prec=prec)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                for _ in range(reps):
                    api.align_all_pairs(z32, prec=prec)
                e1.record(stream)
            torch.cuda.synchronize(dev)
            tms = e0.elapsed_time(e1) / reps
            same = touts[0] == ref32[0]
            tie = ~same & ((touts[2] - ref32[2]).abs() <= 1e-9)
            rel = ((touts[2] - ref32[2]).abs() / ref32[2].abs().clamp(min=1e-300))[same]
            gemm_flop = npairs * 2.0 * (2 * Na) * (2 * Na) * terms
            tc[prec] = {"ms": tms, "ordered_pairs_per_s": Ma * (Ma - 1) / (tms * 1e-3),
                        "speedup_vs_fp64": all_ms / tms, "speedup_vs_mixed": all_mixed_ms / tms,
                        "shift_agreement_with_fp64": float(same.double().mean().item()),
                        "shift_agreement_with_fp64_or_tie": float((same | tie).double().mean().item()),
                        "max_rel_denergy_where_shift_agrees": float(rel.max().item()),
                        "tensor_flop": gemm_flop, "tensor_tflops_over_whole_call":
                            gemm_flop / (tms * 1e-3) / 1e12}
            del touts
        allp["tensor_core"] = {
            "input": "complex64 z; FP64 reference = the FP64 search of the same complex64 input",
            "method": "cross-spectra x DFT matrix as one GEMM (M = 2.1 M pairs, K = 2N, N = 2N "
                      "real columns) on tcgen05, float32 accumulation, top 8 |c|^2 per pair "
                      "re-scored by direct correlation in double-float, theta/energy likewise",
            "variants": tc}
        del za, outs, mouts, z32, ref32

    # uneven batch: 100,000 pairs, n log-uniform in [64, 8192] (multiples of
    # 16), one persistent launch per transform-length bucket with the plan the
    # autotuner chose for it, replayed as a CUDA graph
    rag = None
    if not args.no_ragged:
        from paper_2501_17779_gb300 import synth

        sizes = synth.log_uniform_sizes(SEED + 11, args.ragged_pairs)
        rz1, rz2, roffs = synth.ragged_pairs_device(SEED + 11, sizes, dev)
        Pr = roffs.numel() - 1
        rws = torch.empty(api.ragged_workspace_size(Pr, 8192, local), dtype=torch.uint8, device=dev)
        rout = (torch.empty(Pr, dtype=torch.int32, device=dev),
                torch.empty(Pr, dtype=torch.float64, device=dev),
                torch.empty(Pr, dtype=torch.float64, device=dev),
                torch.empty(Pr, dtype=torch.int8, device=dev))
        with torch.cuda.stream(stream):
            api.align_pairs_ragged(rz1, rz2, roffs, max_n=8192, workspace=rws, out=rout,
                                   autotune=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(3):
                api.align_pairs_ragged(rz1, rz2, roffs, max_n=8192, workspace=rws, out=rout)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        rag_ms = e0.elapsed_time(e1) / 3
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            api.align_pairs_ragged(rz1, rz2, roffs, max_n=8192, workspace=rws, out=rout)
        with torch.cuda.stream(stream):
            graph.replay()
            e0.record(stream)
            for _ in range(3):
                graph.replay()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        rag_graph_ms = e0.elapsed_time(e1) / 3
        fl_rag = ragged_flops(sizes)
        plan = api.ragged_plan(local)
        nz = np.asarray(sizes)
        Lz = np.where(nz & (nz - 1) == 0, nz, 1 << np.ceil(np.log2(2 * nz - 1)).astype(np.int64))
        per_bucket = {}
        for bkt in sorted(set(np.log2(Lz).astype(int).tolist()), reverse=True):
            t_, g_, ms_ = plan[bkt]
            sel = nz[np.log2(Lz).astype(int) == bkt]
            flb = ragged_flops(sel)
            per_bucket[f"L=2^{bkt}"] = {
                "pairs": int(sel.size), "threads": t_,
                "pairs_per_cta": g_ if g_ > 0 else None,
                "ctas_per_pair": -g_ if g_ < 0 else 1, "ms": ms_,
                "frac_of_fp64_peak": (flb / (ms_ * 1e-3) / 1e12 / fp64_peak) if ms_ > 0 else None}
        rag = {"workload": f"{Pr} pairs, n log-uniform in [64, 8192] (multiples of 16), 4..32 "
                           "harmonics, FP64, one persistent launch per transform-length bucket",
               "plans": per_bucket,
               "ms": rag_ms, "graph_ms": rag_graph_ms, "pairs_per_s": Pr / (rag_graph_ms * 1e-3),
               "nodes": int(np.asarray(sizes).sum()),
               "tflops": fl_rag / (rag_graph_ms * 1e-3) / 1e12,
               "frac_of_fp64_peak": fl_rag / (rag_graph_ms * 1e-3) / 1e12 / fp64_peak,
               "status_ok": bool((rout[3] == 0).all().item())}
        del rz1, rz2, roffs, rws, rout, graph

    # elastic shape distance (Sec. 3, Approach 2 with the FFT (t0,R)-step):
    # 4096 pairs of N = 256 gallery curves (50 Fourier-series classes,
    # harmonic perturbation 0.03, random smooth reparameterisation), band 32
    ela = None
    if not args.no_elastic:
        from paper_2501_17779_gb300 import synth

        Ne, Pe, Be = 256, 4096, 32
        ce = torch.from_numpy(synth.shape_gallery(SEED + 13, 2 * Pe, Ne, device=str(dev)).curves).to(dev)
        c1, c2 = ce[:Pe].contiguous(), ce[Pe:].contiguous()
        ews = torch.empty(api.elastic_workspace_size(Pe, Pe, Pe, Ne, Be, local), dtype=torch.uint8,
                          device=dev)
        lms = torch.empty(Pe, dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            eo = api.elastic_distance(c1, c2, band=Be, workspace=ews, lm_steps=lms)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(3):
                api.elastic_distance(c1, c2, band=Be, workspace=ews, out=eo)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ela_ms = e0.elapsed_time(e1) / 3
        el_fl = elastic_flops(lms.cpu().numpy(), eo[3].cpu().numpy(), Ne)
        ela = {"workload": f"{Pe} pairs, N={Ne}, lattice band {Be}, gallery curves (50 classes, "
                           "harmonic perturbation 0.03, random smooth reparameterisation), FP64",
               "ms": ela_ms, "pairs_per_s": Pe / (ela_ms * 1e-3),
               "lm_steps_mean": float(lms.double().mean().item()),
               "roofline": {"bound": "alu", "peak": fp64_peak, "unit": "TFLOP/s",
                            "achieved": el_fl / (ela_ms * 1e-3) / 1e12,
                            "frac": el_fl / (ela_ms * 1e-3) / 1e12 / fp64_peak,
                            "flops_per_launch": el_fl,
                            "count": "FP64 flops counted per refinement step, outer iteration "
                                     "and pair from the kernel's algorithm (bench.py "
                                     "elastic_flops); the float32 lattice programme excluded"},
               "iterations_mean": float(eo[3].double().mean().item()),
               "iterations_max": int(eo[3].max().item()),
               "distance_mean": float(torch.sqrt(eo[2]).mean().item()),
               "status_ok": bool((eo[4] == 0).all().item())}
        del ce, c1, c2, ews, eo

    # k-NN retrieval, 20,000-curve gallery, 1,000 queries, N = 256: the pruning
    # network trained on elastic distances, 200 candidates per query
    knnr = None
    if not args.no_knn:
        from paper_2501_17779_gb300 import knn as knnmod
        from paper_2501_17779_gb300 import synth

        Gk, Qk, Nk, Bk, NC = 20000, 1000, 256, 32, 200
        gal = torch.from_numpy(synth.shape_gallery(SEED + 17, Gk, Nk, device=str(dev)).curves).to(dev)
        qry = torch.from_numpy(synth.shape_gallery(SEED + 19, Qk, Nk, device=str(dev)).curves).to(dev)
        with torch.cuda.stream(stream):
            torch.cuda.synchronize(dev)
            e0.record(stream)
            dg = knnmod.descriptors(gal)
            net, loss, n_train = knnmod.train_pruner(gal, dg, band=Bk, steps=1500, seed=SEED,
                                                     n_near=12, n_rand=4)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            train_ms = e0.elapsed_time(e1)
            e0.record(stream)
            dq = knnmod.descriptors(qry, dg)
            found, _ = knnmod.search(qry, gal, k=10, band=Bk, n_cand=NC, qdesc=dq.x, gdesc=dg.x,
                                     net=net)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            search_ms = e0.elapsed_time(e1)
            Qs = args.knn_exact_queries
            e0.record(stream)
            exact, _ = knnmod.search(qry[:Qs], gal, k=10, band=Bk)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            exact_ms = e0.elapsed_time(e1)
            raw, _ = knnmod.search(qry[:Qs], gal, k=10, band=Bk, n_cand=NC, qdesc=dq.x[:Qs],
                                   gdesc=dg.x)
            torch.cuda.synchronize(dev)
        knnr = {"workload": f"gallery {Gk}, queries {Qk}, N={Nk}, 50 classes, lattice band {Bk}, "
                            f"{NC} candidates per query",
                "queries_per_s": Qk / (search_ms * 1e-3), "search_ms": search_ms,
                "elastic_per_query": NC, "exact_elastic_per_query": Gk,
                "exact_queries_per_s": Qs / (exact_ms * 1e-3),
                "speedup_vs_exact": (exact_ms / Qs) / (search_ms / Qk),
                "recall_at_10": knnmod.recall_at_k(found[:Qs], exact),
                "recall_at_10_raw_descriptors": knnmod.recall_at_k(raw, exact),
                "recall_sample": f"the first {Qs} queries, exact search over all {Gk} curves",
                "train_ms": train_ms, "train_elastic_pairs": n_train, "train_loss": loss,
                "network": "64-256-256-64, bf16 weights, fp32 accumulate, Adam, 1500 steps x 4096 pairs"}
        del gal, qry, dg, dq, found, exact, raw, net

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle

            oracle.build()
            nthreads = os.cpu_count() or 1
            secs, ores = oracle_sample(rp, args.cpu_pairs, N, nthreads)
            n1 = min(128, args.cpu_pairs)
            secs1, _ = oracle_sample(rp, n1, N, 1)
            parity = {"fp64": parity_vs_oracle(ores, ref_shift, ref_theta, ref_energy),
                      "mixed": parity_vs_oracle(ores, *mix_res),
                      "fp32_storage": parity_vs_oracle(ores, sh32, th32, en32,
                                                       zmax=zmax)}
            cpu = {"value": args.cpu_pairs / secs, "unit": "pairs/s", "cores": nthreads,
                   "kind": "oracle", "sample": f"first {args.cpu_pairs} of the 4096 pairs "
                   "(resampling + O(N^2) Kabsch search), one pass, "
                   f"{secs * nthreads:.1f} core-seconds",
                   "single_core": {"value": n1 / secs1, "unit": "pairs/s", "cores": 1,
                                   "sample": f"first {n1} pairs"},
                   "parity_of_gpu_results": parity}
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs": P, "N": N, "curves": C,
                       "input_nodes": int(n_in.sum()), "l2": "inputs larger than L2 "
                       f"({rp.pts.nbytes / 1e6:.0f} MB raw nodes), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof,
            "kernels": kernels,
            "direct": {"align_ms": direct_ms, "pairs_per_s": P / (direct_ms * 1e-3),
                       "fft_align_speedup": direct_ms / al_avg,
                       "end_to_end_speedup": (rs_avg + direct_ms) / (rs_avg + al_avg),
                       "direct_tflops": direct_flops_per_pair(N) * P / (direct_ms * 1e-3) / 1e12},
            "variants": {"fft_mixed": {
                "align_ms": mixed_ms, "pairs_per_s": world * P / ((rs_avg + mixed_ms) * 1e-3),
                "align_speedup_vs_fp64": al_avg / mixed_ms,
                "align_speedup_vs_direct": direct_ms / mixed_ms,
                "shift_agreement_with_fp64": mixed_agree, "disagreements_within_tie": mixed_tie_ok,
                "dtype": "double-float (f32x2) search + f64 c(s*)/theta/energy"},
                "fp32_storage": fp32_storage},
            "all_pairs": allp,
            "ragged": rag,
            "elastic": ela,
            "knn": knnr,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(world, P, 1, e2e_ms), "unit": "pairs/s",
                    "h2d_bytes_per_step": int(rp.pts.nbytes + rp.offsets.nbytes),
                    "d2h_bytes_per_step": int(P * (4 + 8 + 8 + 1)), "ms_per_step": e2e_ms},
            "gpu_launches": 2 * K,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-pairs", type=int, default=4096)
    ap.add_argument("--ref-pairs", type=int, default=512)
    ap.add_argument("--direct-reps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-all-pairs", action="store_true")
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--ragged-pairs", type=int, default=100_000)
    ap.add_argument("--no-elastic", action="store_true")
    ap.add_argument("--no-knn", action="store_true")
    ap.add_argument("--knn-exact-queries", type=int, default=256)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
