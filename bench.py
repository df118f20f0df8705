"""Benchmark of the embedded-ERI transformation (Algorithm 1 of arXiv 1909.08596, section 2.1).

One step = one call of dmet_emb_eri on one embedding problem: orbital checks, the k-AO -> k-EO
half transforms of every needed (k1, k1+q) pair, the Fourier sum to the reference cell, the
contraction over the aux index and the sum over q into the 8-fold packed ERI blocks.

Default workload: the NiO-shaped unrestricted problem (section 3.3's AFM-II NiO cell on the
4x4x4 mesh of section 2.2: 104 AOs and 900 aux functions per cell, 300 embedding orbitals per
spin, alpha-alpha, alpha-beta and beta-beta blocks), with L in the reduced layout (the 1184
(k1, k2) blocks the 8-fold schedule reads, 184 GB) generated on the device from the seeded
generator. The inputs are synthetic stand-ins for the paper's GDF integrals and embedding
orbitals (same shapes, seeded values; synth/lattice.py).

Prints one JSON line. `value` is useful TFLOP/s (the symmetry-reduced algorithmic flop count
of the work the library does) with inputs resident in HBM; `e2e` is the same metric through
the C ABI with host buffers (copies inside the timed region). The headline path is the
split-BF16 tensor-core path; the plain FP64 path is measured alongside where it finishes in
reasonable time. The error of each result against the FP64 CPU oracle is measured on seeded
orbital subsets (exact: an orbital-column subset of the ERI is the method applied to those
columns), per spin block, with L streamed to the oracle in blocks of aux functions.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--workload NAME]
                    [--prec bf16x3|fp64] [--only] [--check-orbitals N]
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
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "embedded-ERI transform TFLOP/s and ms/problem at stated error vs FP64; % of roofline"
DEFAULT_WORKLOAD = "nio_4x4x4_uhf"
SMS = 152
DFMA_PER_SM_CLK = 2  # FP64 FMA lanes per SM per clock on GB300 (1.25 TFLOP/s nominal at 2.07 GHz)
REF_SAMPLE_ORBITALS = 24
# dmet_prec_t codes, and each tensor-core precision's tensor rate relative to dense bf16 (the recipe's
# nominal figures: fp16 = bf16, tf32 = half of bf16); the measured bf16 peak times that ratio is the peak
PREC_CODES = {"fp64": 0, "bf16x3": 1, "tf32": 2, "tf32x3": 3, "fp16x2": 4}
PEAK_RATIO = {"bf16x3": 1.0, "fp16x2": 1.0, "tf32": 0.5, "tf32x3": 0.5}
PREC_DTYPE = {"fp64": "f64", "bf16x3": "bf16x3", "fp16x2": "fp16x2", "tf32": "tf32", "tf32x3": "tf32x3"}
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel class, from an ncu capture:
# (workload, path, kernel class) -> (bytes per launch, digest of the kernel sources at the capture). The
# bytes are the class's DRAM bytes per call over its launches per call (the same per-launch unit as the
# roofline's `achieved`). The roofline reports them only while the sources still have that digest
# (kernel_sources_digest); after any change to the kernels or their job tables, traffic is null.
KERNEL_SOURCES = ["tc_gemm.cuh", "tc_common.cuh", "prec.cuh", "split.cuh", "mixed_impl.cuh", "plan.cu"]
TRAFFIC = {
    # one-pass ncu capture of the contraction launches of one NiO-shaped call with job pacing (aa 526.2 GB,
    # ab 1022.9 GB, bb 529.4 GB read + written) over the class's 5 launches per call
    ("nio_4x4x4_uhf", "bf16x3", "tc_contract"): (2078.5e9 / 5, "9350c8854e55ec2d"),
}


def kernel_sources_digest():
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1909_08596_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(base, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_of(key):
    t = TRAFFIC.get(key)
    return t[0] if t and t[1] == kernel_sources_digest() else None


def schedule_counts(mesh):
    """Per q: the contraction weight (1 for q = -q, 2 for q < -q, 0 for q > -q) and the number of
    transformed k1 (one per orbit {k1, -k1-q}), from their definition (section 2.1's loops with the
    real-orbital symmetries; tests/test_bench_host.py checks them against the library's schedule)."""
    n1, n2, n3 = mesh
    nk = n1 * n2 * n3

    def trip(k):
        return k // (n2 * n3), (k // n3) % n2, k % n3

    def idx(a, b, c):
        return ((a % n1) * n2 + (b % n2)) * n3 + (c % n3)

    neg = [idx(*(-x for x in trip(k))) for k in range(nk)]
    qw, nrep = [], []
    for q in range(nk):
        qw.append(1 if q == neg[q] else (2 if q < neg[q] else 0))
        tq = trip(q)
        cnt = 0
        for k1 in range(nk):
            t1 = trip(k1)
            partner = neg[idx(t1[0] + tq[0], t1[1] + tq[1], t1[2] + tq[2])]
            cnt += k1 <= partner
        nrep.append(cnt)
    return qw, nrep


def useful_flops(spec, n_list, n_aux=None):
    """Algorithmic flops of one problem with the symmetry reductions the library applies.

    Transform (per spin, per computed pair): 8 n_aux (n_ao^2 n + n_ao n^2) (a complex MAC is 8
    flops); contraction: npair (npair+1) K per same-spin block, 2 npair_a npair_b K for
    alpha-beta, K = n_aux * (1 + [q != -q]) summed over the contracted q."""
    qw, nrep = schedule_counts(spec.mesh)
    nao, naux = spec.n_ao, spec.n_aux if n_aux is None else n_aux
    fl_t = 0.0
    K = 0
    for q, w in enumerate(qw):
        if not w:
            continue
        K += naux * (1 if w == 1 else 2)
        for n in n_list:
            fl_t += nrep[q] * 8.0 * naux * (nao * nao * n + nao * n * n)
    pairs = [n * (n + 1) // 2 for n in n_list]
    fl_c = sum(p * (p + 1.0) * K for p in pairs)
    if len(n_list) == 2:
        fl_c += 2.0 * pairs[0] * pairs[1] * K
    return fl_t + fl_c, fl_t, fl_c


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "", 1).isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_spec(base, rank):
    """Weak scaling: every rank transforms its own problem of the same shape (its own seed)."""
    return synth.spec_with(base, seed=base.seed + 17 * rank)


def max_over_ranks(dist, ms, device):
    """The job's time is the slowest rank's (a MAX all-reduce; the only collective, outside the data path)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_ranges(mesh, n_ao, n_emb_list, world):
    """A q shard per rank for splitting one problem over `world` GPUs (strong scaling): contiguous
    ranges of the contracted q (q and -q stay together, as min(q, -q) is the contracted one) whose
    costs (the transforms of the q's representative pairs plus its share of the contraction) are as
    equal as the q granularity allows. Returns [(q_begin, q_end)] covering [0, Nk)."""
    qw, nrep = schedule_counts(mesh)
    nk = len(qw)
    cost = [0.0] * nk
    for q in range(nk):
        if qw[q]:
            cost[q] = sum(nrep[q] * (n_ao * n_ao * n + n_ao * n * n) for n in n_emb_list) + \
                qw[q] * sum(n * n * n * n for n in n_emb_list) / 8.0
    total = sum(cost)
    out, lo, acc = [], 0, 0.0
    for r in range(world - 1):
        target = total * (r + 1) / world
        hi = lo
        while hi < nk and acc + cost[hi] <= target:
            acc += cost[hi]
            hi += 1
        hi = max(hi, lo + 1) if any(cost[lo:]) else hi
        out.append((lo, hi))
        lo = hi
    out.append((lo, nk))
    return out


def sum_over_ranks(dist, tensors):
    """The one exchange step of a q-sharded problem: the FP64 sum of every rank's partial packed ERI
    blocks (Algorithm 1's sum over the aux momentum, split across ranks), in place on every rank."""
    if not dist:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors


def job_tflops(world, flops_per_problem, steps, ms_total):
    """Whole-job throughput: every rank's problems over the slowest rank's time."""
    return world * flops_per_problem * steps / (ms_total / 1e3) / 1e12


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def subset_orbitals(spec, n_sub, seed=0):
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(spec.n_emb, min(n_sub, spec.n_emb), replace=False)) for _ in range(spec.n_spin)]


def s8_positions(S):
    """Packed 8-fold indices of every (ij|kl) with i, j, k, l in the orbital subset S."""
    i, j, k, l = np.meshgrid(*([np.arange(len(S))] * 4), indexing="ij")
    ii, jj, kk, ll = S[i.ravel()], S[j.ravel()], S[k.ravel()], S[l.ravel()]
    I, J = np.maximum(ii, jj), np.minimum(ii, jj)
    K_, L_ = np.maximum(kk, ll), np.minimum(kk, ll)
    a, b = I * (I + 1) // 2 + J, K_ * (K_ + 1) // 2 + L_
    P, Q = np.maximum(a, b), np.minimum(a, b)
    return P * (P + 1) // 2 + Q


def ab_positions(Sa, Sb, nb):
    """Indices [IJ][KL] of the alpha-beta block for i, j in Sa (alpha) and k, l in Sb (beta)."""
    i, j, k, l = np.meshgrid(np.arange(len(Sa)), np.arange(len(Sa)), np.arange(len(Sb)), np.arange(len(Sb)),
                             indexing="ij")
    ii, jj, kk, ll = Sa[i.ravel()], Sa[j.ravel()], Sb[k.ravel()], Sb[l.ravel()]
    I, J = np.maximum(ii, jj), np.minimum(ii, jj)
    K_, L_ = np.maximum(kk, ll), np.minimum(kk, ll)
    npb = nb * (nb + 1) // 2
    return (I * (I + 1) // 2 + J) * npb + (K_ * (K_ + 1) // 2 + L_)


def block_positions(spec, S):
    """Per output block b: the packed positions of the subset tensor (i j | k l), C order."""
    if spec.n_spin == 1:
        return [s8_positions(S[0])]
    return [s8_positions(S[0]), ab_positions(S[0], S[1], spec.n_emb), s8_positions(S[1])]


def block_spins(spec):
    return [(0, 0)] if spec.n_spin == 1 else [(0, 0), (0, 1), (1, 1)]


def error_stats(got, ref):
    d = got - ref
    return {"rel_fro": float(np.linalg.norm(d) / np.linalg.norm(ref)), "max_abs": float(np.abs(d).max()),
            "max_abs_over_max": float(np.abs(d).max() / np.abs(ref).max()), "rms": float(np.sqrt(np.mean(d * d)))}


def run_reference(args):
    """The reference arm: the CPU oracle (Algorithm 1 as written, every q and every k1, dense
    contraction; L streamed over aux functions) on a bounded sample of the workload, on the host
    cores. Uses only synth (host generator) and oracle; never the library under test."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    spec = synth.CONFIGS[args.workload]
    # sample: REF_SAMPLE_ORBITALS orbitals per spin, the first p_ref aux functions (the host generator
    # draws about 7.5e6 normals per second, so the sample's L is drawn in about 10 s at most)
    per_p = (spec.n_ao * spec.nk) ** 2
    p_ref = int(max(1, min(spec.n_aux, 75_000_000 // per_p)))
    Lb = synth.fourier_L(synth.real_space_B(spec, 0, p_ref), spec.mesh)
    _, Cs, _ = synth.make_problem(spec, with_L=False)
    S = subset_orbitals(spec, REF_SAMPLE_ORBITALS)
    Csub = [np.ascontiguousarray(C[:, :, s]) for C, s in zip(Cs, S)]
    n_list = [len(s) for s in S]
    fl = useful_flops(spec, n_list, n_aux=p_ref)[0]
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.embedded_eri_pblocks([Lb], Csub, spec.mesh)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    sec = float(np.mean(times))
    value = fl / sec / 1e12
    sample = (f"Algorithm 1 (all q, all k1, dense contraction) on {n_list[0]} of {spec.n_emb} embedding orbitals "
              f"per spin and the first {p_ref} of {spec.n_aux} aux functions per step; useful flops of that "
              f"sub-problem")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(spec, "fp64"),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(spec, prec, layout=None):
    return {"workload": spec.name, "mesh": list(spec.mesh), "n_ao": spec.n_ao, "n_aux": spec.n_aux,
            "n_emb": spec.n_emb, "n_spin": spec.n_spin, "prec": prec, "pack": "s8",
            **({"l_layout": layout} if layout else {})}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def roofline(spec, prec, kstats, sustained=False):
    peaks, peak_src = measured_peaks()
    top = max(kstats, key=lambda k: k["ms"])
    avg_ms = top["ms"] / max(top["launches"], 1)
    if prec == "fp64":
        peak = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
        achieved = top["flops"] / (top["ms"] / 1e3) / 1e12 if top["ms"] > 0 else 0.0
        return {"bound": "alu", "kernel": top["name"], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_of((spec.name, prec, top["name"])),
                "flops_counted": "algorithmic FP64 flops",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (FP64 runs on the CUDA cores)",
                "avg_launch_ms": avg_ms}
    # A tensor kernel's roofline is whichever of its two floors is higher: executed tensor flops at
    # the precision's peak (the measured bf16 peak times the nominal ratio), or its algorithmic bytes
    # at the measured HBM copy rate.
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    peak_t, peak_b = peaks[key] * PEAK_RATIO[prec], peaks["hbm_gbs"]
    secs = top["ms"] / 1e3 / max(top["launches"], 1)
    fl_l = top["exec_flops"] / max(top["launches"], 1)
    by_l = top["bytes"] / max(top["launches"], 1)
    t_tensor, t_hbm = fl_l / (peak_t * 1e12), by_l / (peak_b * 1e9)
    tensor = {"achieved": fl_l / secs / 1e12 if secs > 0 else 0.0, "peak": peak_t, "unit": "TFLOP/s"}
    hbm = {"achieved": by_l / secs / 1e9 if secs > 0 else 0.0, "peak": peak_b, "unit": "GB/s"}
    for d in (tensor, hbm):
        d["frac"] = d["achieved"] / d["peak"]
    tensor["frac_of_burst_peak"] = tensor["achieved"] / (peaks["bf16_tflops"] * PEAK_RATIO[prec])
    main, other = (hbm, tensor) if t_hbm > t_tensor else (tensor, hbm)
    useful = top["flops"] / (top["ms"] / 1e3) / 1e12 if top["ms"] > 0 else 0.0
    return {"bound": "hbm" if main is hbm else "tensor", "kernel": top["name"], **main,
            "traffic": traffic_of((spec.name, prec, top["name"])),
            "other_bound": {"bound": "tensor" if main is hbm else "hbm", **other},
            "flops_counted": "executed tensor flops (every slice product issued, whole tiles)",
            "bytes_counted": "algorithmic bytes per launch: operands read once, result written once",
            "useful_achieved_tflops": useful, "useful_frac": useful / peak_t,
            "peak_source": f"{peak_src} {key} x {PEAK_RATIO[prec]} ({prec}) and hbm_gbs"
                           + (" (sustained: the step runs the kernels for seconds under the power cap)" if sustained
                              else " (burst: a short step)"), "avg_launch_ms": avg_ms}


def kernel_table(kstats):
    tot_ms = max(sum(x["ms"] for x in kstats), 1e-9)
    kernels = {}
    for k in kstats:
        if not k["launches"]:
            continue
        e = {"launches": k["launches"], "ms": round(k["ms"], 3), "share": round(k["ms"] / tot_ms, 4)}
        if k["ms"] > 0 and k["bytes"] > 0:
            e["hbm_gbs"] = round(k["bytes"] / (k["ms"] / 1e3) / 1e9, 1)  # algorithmic bytes / time
        if k["ms"] > 0 and k["exec_flops"] > 0:
            e["exec_tflops"] = round(k["exec_flops"] / (k["ms"] / 1e3) / 1e12, 1)
        if k["ms"] > 0 and k["flops"] > 0:
            e["useful_tflops"] = round(k["flops"] / (k["ms"] / 1e3) / 1e12, 1)
        kernels[k["name"]] = e
    return kernels


def measure(dm, torch, spec, desc, Ld, Cd, outs, steps, args, dist, world, local, ws_limit, autotune,
            qshard=False):
    """Times `steps` calls of dmet_emb_eri on resident inputs (CUDA events on the plan's stream). With
    qshard, every rank computes its q shard of one problem and each step ends with the FP64 sum of the
    partial ERI blocks over the ranks (NCCL), inside the timed region."""
    n_list = [spec.n_emb] * spec.n_spin
    fl_total, fl_t, fl_c = useful_flops(spec, n_list)
    stream = torch.cuda.current_stream()
    plan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream, workspace_limit=ws_limit)
    try:
        tile_widths = None
        if autotune:
            # Tile widths of the transform GEMMs chosen by timing (outside the timed region).
            dm.dmet_emb_autotune(plan, [Ld], [Cd], [outs])
            tile_widths = dm.dmet_emb_tile_widths(plan, 0)

        def step():
            dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
            if qshard:
                sum_over_ranks(dist, outs)

        for _ in range(args.warmup):
            step()
        st, stats = dm.dmet_emb_status(plan, 0)
        if st != dm.binding.DMET_OK:
            raise RuntimeError(f"device status {st}: {dm.dmet_emb_last_error()} {stats}")
        dm.dmet_emb_profile(plan, True)
        launches0 = dm.dmet_emb_launch_count(plan)
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop()
        ms_total = ev0.elapsed_time(ev1)
        launches = dm.dmet_emb_launch_count(plan) - launches0
        kstats = [dm.dmet_emb_profile_read(plan, k) for k in range(dm.dmet_emb_profile_count())]
        dm.dmet_emb_profile(plan, False)
        st, stats = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    ms_total = max_over_ranks(dist, ms_total, "cuda")
    ms_step = ms_total / steps
    prec = {v: k for k, v in PREC_CODES.items()}[desc.prec]
    return {
        "value": job_tflops(1 if qshard else world, fl_total, steps, ms_total), "ms_per_step": ms_step,
        "useful_tflop_per_problem": fl_total / 1e12,
        "useful_split": {"transform": fl_t / 1e12, "contraction": fl_c / 1e12},
        # a step of a second or more runs the kernels for seconds under the power cap: the sustained peak
        "roofline": roofline(spec, prec, kstats, sustained=ms_step >= 1000.0), "kernels": kernel_table(kstats),
        "gpu_launches": int(launches),
        "clocks": clk, "steps": steps, "tile_widths": tile_widths,
        "device_checks": {"status": int(st), "orthonormality": stats[0], "realness": stats[1],
                          "hermiticity_L": stats[2], "time_reversal_L": stats[3]},
    }


def gather_subsets(torch, outs, positions):
    """The GPU's packed values at the subset positions of every block (gathered on the device)."""
    return [outs[b][torch.as_tensor(pos, device=outs[b].device)].cpu().numpy() for b, pos in enumerate(positions)]


def measure_fock_and_bath(dm, torch, spec, Cd, eri0):
    """The embedding one-particle Hamiltonian from this ERI (dmet_emb_fock) and the DMET bath that
    produces such orbitals (dmet_emb_bath), FP64 kernels, timed on their own (restricted problems)."""
    stream = torch.cuda.current_stream()
    desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb)
    plan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream, workspace_limit=16 << 30)
    fock = bath = None
    try:
        Fk = torch.from_numpy(synth.fock_k(synth.real_space_fock(spec), spec.mesh)).cuda()
        gam = torch.from_numpy(synth.embedding_density(spec.n_emb, spec.seed)).cuda()
        fo = torch.empty((spec.n_emb, spec.n_emb), dtype=torch.float64, device="cuda")
        if spec.n_emb <= 232:
            for _ in range(3):
                dm.dmet_emb_fock(plan, Fk, Cd[0], eri0, gam, fo)
            dm.dmet_emb_profile(plan, True)
            reps = 10
            ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ef0.record(stream)
            for _ in range(reps):
                dm.dmet_emb_fock(plan, Fk, Cd[0], eri0, gam, fo)
            ef1.record(stream)
            torch.cuda.synchronize()
            fk = [k for k in (dm.dmet_emb_profile_read(plan, i) for i in range(dm.dmet_emb_profile_count()))
                  if k["name"] == "embedding_fock"][0]
            dm.dmet_emb_profile(plan, False)
            f_ms = ef0.elapsed_time(ef1) / reps
            f_peak = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
            f_tf = fk["flops"] / reps / (f_ms / 1e3) / 1e12
            fock = {"ms": f_ms, "launches_per_call": fk["launches"] // reps,
                    "roofline": {"bound": "alu", "achieved": f_tf, "peak": f_peak, "unit": "TFLOP/s",
                                 "frac": f_tf / f_peak,
                                 "flops_counted": "FP64 flops the kernels execute (transform GEMMs; 2 n^2 exchange "
                                                  "and n(n+1)/2 Coulomb multiply-adds per ERI pair row)",
                                 "peak_source": "derived FP64 peak (152 SMs x 2 FMA/clk x 2 x 2070 MHz)"}}
    finally:
        dm.dmet_emb_destroy(plan)
    # The bath: the same cell and mesh, its n_AO LOs as the impurity and 8 of them as the valence
    # columns of the SVD (the valence shell of a two-atom s/p cell), from a synthetic gapped mean field.
    if spec.nk > 1:
        n_val = min(8, spec.n_ao)
        bspec = synth.spec_with(spec, n_emb=spec.n_ao + n_val)
        h = synth.mean_field_hamiltonian(bspec, spec.n_ao // 2)
        gk = torch.from_numpy(synth.mean_field_density(h, spec.mesh, spec.n_ao // 2)).cuda()
        Ulo = torch.from_numpy(synth.lo_rotation(bspec)).cuda()
        val = list(range(0, spec.n_ao, max(1, spec.n_ao // n_val)))[:n_val]
        Cb = torch.empty((spec.nk, spec.n_ao, bspec.n_emb), dtype=torch.complex128, device="cuda")
        binfo = torch.zeros(n_val + 5, dtype=torch.float64, device="cuda")
        bplan = dm.dmet_emb_plan(dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, bspec.n_emb),
                                 stream=stream.cuda_stream, workspace_limit=1 << 30)
        try:
            for _ in range(3):
                dm.dmet_emb_bath(bplan, gk, Ulo, val, Cb, binfo)
            reps = 10
            eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            eb0.record(stream)
            for _ in range(reps):
                dm.dmet_emb_bath(bplan, gk, Ulo, val, Cb, binfo)
            eb1.record(stream)
            torch.cuda.synchronize()
            bi = binfo.cpu().numpy()
            bath = {"ms": eb0.elapsed_time(eb1) / reps, "n_lo": spec.n_ao, "n_val": n_val,
                    "launches_per_call": dm.dmet_emb_launch_count(bplan) // (reps + 3),
                    "jacobi_sweeps": int(bi[n_val + 2]), "sigma_min_over_max": float(bi[n_val + 4])}
        finally:
            dm.dmet_emb_destroy(bplan)
    return fock, bath


def measure_e2e(dm, torch, desc, holder, Cs, positions, fl_total, world, args, ws_limit):
    """End to end through the C ABI with host buffers: every step copies the (k1, k2) blocks of L the
    schedule reads and C from pinned host memory to the device, runs the call and reads the ERI blocks
    back. A plan of its own, built with the q-block size capped (DMET_QBLOCK) so that L streams in
    small blocks. holder["Ld"] (the device L) is released once its host copy exists."""
    Ld = holder["Ld"]
    Lh = torch.empty(Ld.shape, dtype=Ld.dtype, pin_memory=True)
    Lh.copy_(Ld)
    holder["Ld"] = None
    del Ld
    torch.cuda.empty_cache()
    Ch = [torch.from_numpy(c).pin_memory() for c in Cs]
    nblk = 1 if desc.n_spin == 1 else 3
    Oh = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64).pin_memory() for b in range(nblk)]
    stream = torch.cuda.current_stream()
    old_qb = os.environ.get("DMET_QBLOCK")
    if args.e2e_qblock > 0:
        os.environ["DMET_QBLOCK"] = str(args.e2e_qblock)
    try:
        eplan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream, workspace_limit=ws_limit)
    finally:
        if old_qb is None:
            os.environ.pop("DMET_QBLOCK", None)
        else:
            os.environ["DMET_QBLOCK"] = old_qb
    try:
        dm.dmet_emb_eri(eplan, [Lh], [Ch], [Oh])  # warm-up (allocates the staging buffers)
        torch.cuda.synchronize()
        dm.dmet_emb_profile(eplan, False)  # clears the counters (no events are recorded)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            dm.dmet_emb_eri(eplan, [Lh], [Ch], [Oh])
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        copy_b = sum(k["bytes"] for k in (dm.dmet_emb_profile_read(eplan, i)
                                          for i in range(dm.dmet_emb_profile_count()))
                     if k["name"] == "host_copy") / args.e2e_steps
        st, _ = dm.dmet_emb_status(eplan, 0)
    finally:
        dm.dmet_emb_destroy(eplan)
    d2h_b = int(sum(o.numel() * 8 for o in Oh))
    sub = [Oh[b].numpy()[pos] for b, pos in enumerate(positions)]
    return {"value": world * fl_total / e2e_s / 1e12, "unit": "TFLOP/s",
            "h2d_bytes_per_step": int(copy_b) - d2h_b, "d2h_bytes_per_step": d2h_b,
            "host_L_bytes": int(Lh.numel() * 16), "ms_per_step": e2e_s * 1e3, "steps": args.e2e_steps,
            "qblock_cap": args.e2e_qblock, "status": int(st)}, sub


def oracle_check(torch, spec, Cs, S, p_block, baseline_s=12.0):
    """The FP64 oracle's (ij|kl) on the orbital subsets S, per spin block (the real part, in the order of
    block_positions), with every aux function's L streamed to the oracle from the device generator
    P-block by P-block; plus the oracle's own rate on the first blocks (about baseline_s seconds) as
    the CPU baseline."""
    import oracle
    from synth import gpu as sgpu
    Csub = [np.ascontiguousarray(C[:, :, s]) for C, s in zip(Cs, S)]
    n_list = [len(s) for s in S]
    acc = None
    t_oracle, p_timed, t_base, p_base = 0.0, 0, None, 0
    gen_check = None
    t_all = time.perf_counter()
    for p0 in range(0, spec.n_aux, p_block):
        p1 = min(spec.n_aux, p0 + p_block)
        blk = sgpu.L_blocks_device(torch, spec, p0, p1).cpu().numpy()
        torch.cuda.empty_cache()
        if gen_check is None:
            # the device generator against the host one on this block's first aux function
            h = synth.fourier_L(synth.real_space_B(spec, p0, p0 + 1), spec.mesh)
            gen_check = float(np.abs(blk[:, :, :1] - h).max() / np.abs(h).max())
        t0 = time.perf_counter()
        part = oracle.embedded_eri_pblocks([blk], Csub, spec.mesh)
        t_oracle += time.perf_counter() - t0
        p_timed += p1 - p0
        if t_base is None and t_oracle >= baseline_s:
            t_base, p_base = t_oracle, p_timed
        if acc is None:
            acc = part
        else:
            for k in acc:
                acc[k] += part[k]
        del blk
    if t_base is None:
        t_base, p_base = t_oracle, p_timed
    refs = [acc[k].real.ravel() for k in block_spins(spec)]
    imag = max(float(np.abs(acc[k].imag).max() / np.abs(acc[k].real).max()) for k in block_spins(spec))
    fl_base = useful_flops(spec, n_list, n_aux=p_base)[0]
    base = {"value": fl_base / t_base / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"Algorithm 1 (all q, all k1, dense contraction; L streamed over aux functions) on {n_list[0]} "
                      f"of {spec.n_emb} embedding orbitals per spin and the first {p_base} of {spec.n_aux} aux "
                      f"functions ({t_base:.1f} s); useful flops of that sub-problem"}
    return refs, base, {"oracle_s": t_oracle, "wall_s": time.perf_counter() - t_all,
                        "device_vs_host_generator_max_rel": gen_check, "oracle_max_imag_over_max": imag}


def run_batch(args):
    """48 uneven problems in one plan, replayed from a CUDA graph: problems/s and the p50/p99
    per-problem device latency of the split-BF16 path as grouped persistent launches (the default
    batch mode) and with each problem on its own side stream, and of the FP64 path."""
    print(json.dumps(batch_line(args)), flush=True)
    return 0


def batch_line(args, arms=("bf16x3", "bf16x3_streams", "fp64")):
    """The batch48 measurement (see run_batch) over the given arms, as one JSON-able dict."""
    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    libbuild.build()
    specs = synth.batch_specs(48)
    probs = []
    for sp in specs:
        L, Cs, _ = synth.make_problem(sp)
        probs.append((sp, L, Cs))
    Ls = [torch.from_numpy(L).cuda() for _, L, _ in probs]
    Cds = [[torch.from_numpy(c).cuda() for c in C] for _, _, C in probs]
    stream = torch.cuda.Stream()
    out = {}
    results = {}
    for arm in arms:
        prec = "fp64" if arm == "fp64" else "bf16x3"
        pcode = dm.binding.DMET_PREC_FP64 if prec == "fp64" else dm.binding.DMET_PREC_BF16X3
        descs = [dm.make_desc(sp.mesh, sp.n_ao, sp.n_aux, sp.n_emb, n_spin=sp.n_spin, prec=pcode) for sp in specs]
        outs = [[torch.empty(dm.dmet_emb_eri_bytes(d, b) // 8, dtype=torch.float64, device="cuda")
                 for b in range(1 if d.n_spin == 1 else 3)] for d in descs]
        with torch.cuda.stream(stream):
            plan = dm.dmet_emb_plan(descs, stream=stream.cuda_stream, workspace_limit=64 << 30)
            grouped = dm.dmet_emb_batch_mode(plan, 1 if arm == "bf16x3" else 0)
            if prec != "fp64" and not args.no_autotune:
                dm.dmet_emb_autotune(plan, Ls, Cds, outs)
            # per-problem device latency from one profiled (non-graph) call
            dm.dmet_emb_profile(plan, True)
            dm.dmet_emb_eri(plan, Ls, Cds, outs)
            lat = sorted(dm.dmet_emb_problem_ms(plan, p) for p in range(len(specs)))
            kern = kernel_table([dm.dmet_emb_profile_read(plan, k) for k in range(dm.dmet_emb_profile_count())])
            dm.dmet_emb_profile(plan, False)
            dm.dmet_emb_graph(plan, True)
            for _ in range(args.warmup):
                dm.dmet_emb_eri(plan, Ls, Cds, outs)
            steps = args.steps if prec != "fp64" else min(args.steps, args.fp64_steps if args.fp64_steps > 0 else 3)
            l0 = dm.dmet_emb_launch_count(plan)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                dm.dmet_emb_eri(plan, Ls, Cds, outs)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / steps
            launches = dm.dmet_emb_launch_count(plan) - l0
            st = [dm.dmet_emb_status(plan, p)[0] for p in range(len(specs))]
            dm.dmet_emb_destroy(plan)
        fl = sum(useful_flops(sp, [sp.n_emb] * sp.n_spin)[0] for sp in specs)
        out[arm] = {"problems_per_s": len(specs) / (ms / 1e3), "ms_per_batch": ms, "useful_tflops": fl / (ms / 1e3) / 1e12,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "latency": "batch completion (every problem ends with the last grouped launch)" if grouped
                    else "per problem on its side stream",
                    "grouped_launches": bool(grouped), "gpu_launches_per_batch": int(launches) // max(steps, 1),
                    "all_ok": all(x == 0 for x in st), "steps": steps,
                    "kernels_profiled_call": kern}
        results[arm] = [[o.cpu().numpy() for o in row] for row in outs]
    # errors vs the oracle on 8-orbital subsets of every problem (alpha block)
    import oracle
    errs = {p: [] for p in results}
    rng = np.random.default_rng(0)
    for i, (sp, L, Cs) in enumerate(probs):
        S = np.sort(rng.choice(sp.n_emb, min(8, sp.n_emb), replace=False))
        eri = oracle.embedded_eri(L, np.ascontiguousarray(Cs[0][:, :, S]), sp.mesh).real.ravel()
        pos = s8_positions(S)
        for p in results:
            g = results[p][i][0][pos]
            errs[p].append(float(np.linalg.norm(g - eri) / np.linalg.norm(eri)))
    for p in errs:
        out[p]["max_rel_fro_vs_oracle"] = max(errs[p])
    line = {"metric": METRIC, "workload": "batch48 (48 uneven problems)", "value": out["bf16x3"]["useful_tflops"],
            "unit": "TFLOP/s", "problems": len(specs), **{p: out[p] for p in out}}
    if "fp64" in out:
        line["speedup_bf16x3_over_fp64"] = out["fp64"]["ms_per_batch"] / out["bf16x3"]["ms_per_batch"]
    if "bf16x3_streams" in out:
        line["speedup_grouped_over_streams"] = out["bf16x3_streams"]["ms_per_batch"] / out["bf16x3"]["ms_per_batch"]
    return line


def _ws_estimate(sp, bq=2):
    """Rough device workspace of one split-BF16 problem at q-block bq (the contraction operands, the
    q-block's transform operands), used only to form resident groups; the plan has the last word."""
    nk, nao, naux, n = sp.nk, sp.n_ao, sp.n_aux, sp.n_emb
    npair = n * (n + 1) // 2
    xt = 6 * npair * nk * naux * sp.n_spin
    a2 = 6 * bq * naux * n * (nk + 2) * nao
    ls = 6 * bq * (nk // 2 + 1) * naux * nao * 2 * nao
    zt = bq * naux * n * 2 * n * 8
    return int(1.25 * (xt + a2 + ls + zt)) + (256 << 20)


def resident_groups(needs, budget):
    """Consecutive problems packed into groups whose summed device need stays within budget (a
    problem larger than the budget alone forms its own group)."""
    groups, cur, used = [], [], 0
    for i, need in enumerate(needs):
        if cur and used + need > budget:
            groups.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += need
    if cur:
        groups.append(cur)
    return groups


def run_batch_stated(args):
    """The batched workload at its stated size ranges (n_AO 26..104, n_aux = 8.5 n_AO, n_emb 40..300,
    Nk in {8, 27, 36, 64}, half unrestricted; 48 problems, ~0.9 TB of reduced L in total): too large
    to hold at once, it runs as resident groups, each one plan in grouped mode (its L generated on
    the device, then one warm-up call and one timed call replayed from a graph). problems/s = 48 over
    the sum of the groups' timed calls; a problem's latency is its group's call."""
    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    from synth import gpu as sgpu
    libbuild.build()
    os.environ.setdefault("DMET_QBLOCK", "2")
    specs = synth.batch_specs(48, n_ao_range=(26, 104), n_emb_range=(40, 300))
    pcode = dm.binding.DMET_PREC_BF16X3
    descs = [dm.make_desc(sp.mesh, sp.n_ao, sp.n_aux, [sp.n_emb] * sp.n_spin if sp.n_spin == 2 else sp.n_emb,
                          n_spin=sp.n_spin, prec=pcode, l_layout=1) for sp in specs]
    pairs = [dm.dmet_emb_l_pairs(d) for d in descs]
    lbytes = [len(pr) * sp.n_aux * sp.n_ao ** 2 * 16 for pr, sp in zip(pairs, specs)]
    obytes = [sum(dm.dmet_emb_eri_bytes(d, b) for b in range(1 if d.n_spin == 1 else 3)) for d in descs]
    free, _ = torch.cuda.mem_get_info()
    groups = resident_groups([lbytes[i] + obytes[i] + _ws_estimate(sp) for i, sp in enumerate(specs)],
                             free - (12 << 30))
    # the three smallest problems are checked against the oracle (8-orbital subsets)
    check_ids = sorted(range(len(specs)), key=lambda i: lbytes[i])[:3]
    stream = torch.cuda.Stream()
    total_ms, gen_s, lat, launches, all_ok, active_all = 0.0, 0.0, [], 0, True, True
    outs_check = {}
    group_ms = []
    with torch.cuda.stream(stream):
        for g in groups:
            t0 = time.perf_counter()
            Ls = [sgpu.make_L_pairs_device(torch, specs[i], pairs[i]) for i in g]
            Cds = [[torch.from_numpy(c).cuda() for c in synth.make_problem(specs[i], with_L=False)[1]] for i in g]
            outs = [[torch.empty(dm.dmet_emb_eri_bytes(descs[i], b) // 8, dtype=torch.float64, device="cuda")
                     for b in range(1 if descs[i].n_spin == 1 else 3)] for i in g]
            torch.cuda.synchronize()
            gen_s += time.perf_counter() - t0
            ws_free = torch.cuda.mem_get_info()[0] - (4 << 30)
            plan = dm.dmet_emb_plan([descs[i] for i in g], stream=stream.cuda_stream, workspace_limit=ws_free)
            try:
                active = dm.dmet_emb_batch_mode(plan, 1)
                active_all &= active or len(g) == 1
                dm.dmet_emb_graph(plan, True)
                dm.dmet_emb_eri(plan, Ls, Cds, outs)
                l0 = dm.dmet_emb_launch_count(plan)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dm.dmet_emb_eri(plan, Ls, Cds, outs)
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1)
                launches += dm.dmet_emb_launch_count(plan) - l0
                all_ok &= all(dm.dmet_emb_status(plan, p)[0] == 0 for p in range(len(g)))
            finally:
                dm.dmet_emb_destroy(plan)
            total_ms += ms
            group_ms.append(ms)
            lat += [ms] * len(g)
            for j, i in enumerate(g):
                if i in check_ids:
                    outs_check[i] = outs[j][0].cpu().numpy()
            del Ls, Cds, outs
            torch.cuda.empty_cache()
    import oracle
    errs = []
    rng = np.random.default_rng(0)
    for i in check_ids:
        sp = specs[i]
        L, Cs, _ = synth.make_problem(sp)
        S = np.sort(rng.choice(sp.n_emb, 8, replace=False))
        eri = oracle.embedded_eri(L, np.ascontiguousarray(Cs[0][:, :, S]), sp.mesh).real.ravel()
        g_ = outs_check[i][s8_positions(S)]
        errs.append(float(np.linalg.norm(g_ - eri) / np.linalg.norm(eri)))
    fl = sum(useful_flops(sp, [sp.n_emb] * sp.n_spin)[0] for sp in specs)
    line = {"metric": METRIC, "workload": "batch48_stated (48 uneven problems at the stated size ranges)",
            "value": fl / (total_ms / 1e3) / 1e12, "unit": "TFLOP/s", "problems": len(specs),
            "problems_per_s": len(specs) / (total_ms / 1e3), "ms_per_batch": total_ms,
            "useful_tflop_per_batch": fl / 1e12, "groups": [len(g) for g in groups], "group_ms": group_ms,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "latency": "the call of the problem's resident group (grouped launches: every problem of a group ends with it)",
            "grouped_launches": bool(active_all), "gpu_launches_per_batch": int(launches), "all_ok": bool(all_ok),
            "l_bytes_total": int(sum(lbytes)), "input_generation_s": gen_s, "dtype": "bf16x3",
            "max_rel_fro_vs_oracle": max(errs), "checked": [specs[i].name for i in check_ids],
            "check": "8-orbital subsets of the three smallest problems (alpha block) against the CPU oracle",
            "fp64": "not run at these sizes: 1613 TFLOP of useful work per batch at the FP64 pipe's 1.26 TFLOP/s "
                    "is over 20 minutes (the narrowed batch48 line compares the two paths)"}
    print(json.dumps(line), flush=True)
    return 0


def run_complex(args):
    """The h-BN-shaped problem (config 1's sizes) with general complex embedding orbitals (sym = NONE,
    dense complex ERI): the tensor-core path against the FP64 path, on resident inputs, with 4000
    sampled (ij|kl) checked against the CPU oracle's per-q factors."""
    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    libbuild.build()
    spec = synth.CONFIGS["hbn_6x6x1"]
    n, nk, naux, nao = spec.n_emb, spec.nk, spec.n_aux, spec.n_ao
    L = synth.make_L(spec)
    C = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec), spec.mesh)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(C).cuda()]
    out = torch.empty(n ** 4, dtype=torch.complex128, device="cuda")
    # useful flops: every (k1, k1 + q) pair's two half transforms; the contraction over every q with
    # (ij|kl) counted for kl <= ij ((kl|ij) = (ij|kl)), 8 flops per complex multiply-add
    fl_t = nk * nk * 8.0 * naux * (nao * nao * n + nao * n * n)
    fl_c = 4.0 * n * n * (n * n + 1.0) * naux * nk
    rng = np.random.default_rng(5)
    idx = rng.integers(0, n, size=(4000, 4))
    import oracle
    Lq = oracle.embedded_3idx(L, C, spec.mesh)
    ref = oracle.eri_entries(Lq, Lq, spec.mesh, idx)
    stream = torch.cuda.Stream()
    res = {}
    for prec in ("bf16x3", "fp64"):
        d = dm.make_desc(spec.mesh, nao, naux, n, sym=dm.binding.DMET_SYM_NONE, eri_pack=dm.binding.DMET_PACK_FULL,
                         prec=PREC_CODES[prec])
        steps = args.steps if prec != "fp64" else 1
        with torch.cuda.stream(stream):
            plan = dm.dmet_emb_plan(d, stream=stream.cuda_stream)
            try:
                for _ in range(args.warmup if prec != "fp64" else 1):
                    dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
                dm.dmet_emb_profile(plan, True)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / steps
                kern = kernel_table([dm.dmet_emb_profile_read(plan, k) for k in range(dm.dmet_emb_profile_count())])
                st = dm.dmet_emb_status(plan, 0)[0]
            finally:
                dm.dmet_emb_destroy(plan)
        got = out.cpu().numpy().reshape(n, n, n, n)[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
        res[prec] = {"ms_per_call": ms, "useful_tflops": (fl_t + fl_c) / (ms / 1e3) / 1e12, "status": st,
                     "rel_fro_sampled": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                     "max_abs_over_max_sampled": float(np.abs(got - ref).max() / np.abs(ref).max()),
                     "kernels": kern, "steps": steps}
    line = {"metric": METRIC, "workload": "hbn_6x6x1_complex (general complex orbitals, dense complex ERI)",
            "value": res["bf16x3"]["useful_tflops"], "unit": "TFLOP/s", "dtype": "bf16x3",
            "useful_tflop_per_call": (fl_t + fl_c) / 1e12, **res,
            "speedup_bf16x3_over_fp64": res["fp64"]["ms_per_call"] / res["bf16x3"]["ms_per_call"]}
    print(json.dumps(line), flush=True)
    return 0


def run_shard_emulation(args):
    """The q-shard split of one problem (the multi-GPU path of `--multi qshard`) run shard after shard on
    this one GPU: each shard is the plan of one rank (its q range, its blocks of the reduced L), timed on
    its own; the FP64 sum of the shards' partial ERI blocks is compared with the unsharded call. The
    shards never wait on one another. What a multi-GPU run adds, the sum-reduce of the ERI blocks over
    NCCL, is not measured here: its bytes are reported."""
    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    from synth import gpu as sgpu
    libbuild.build()
    spec = synth.CONFIGS[args.workload]
    n_list = [spec.n_emb] * spec.n_spin
    nshard = args.emulate_shards
    ranges = shard_ranges(spec.mesh, spec.n_ao, n_list, nshard)
    _, Cs, _ = synth.make_problem(spec, with_L=False)
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    pcode = PREC_CODES[args.prec]
    layout = dm.binding.DMET_L_REDUCED
    stream = torch.cuda.current_stream()

    def one(q_range, outs):
        d = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, n_spin=spec.n_spin, l_layout=layout,
                         q_range=q_range, prec=pcode)
        Ld = sgpu.make_L_pairs_device(torch, spec, dm.dmet_emb_l_pairs(d))
        torch.cuda.synchronize()
        plan = dm.dmet_emb_plan(d, stream=stream.cuda_stream, workspace_limit=torch.cuda.mem_get_info()[0] - (2 << 30))
        try:
            dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
            e1.record(stream)
            stream.synchronize()
            st = dm.dmet_emb_status(plan, 0)[0]
        finally:
            dm.dmet_emb_destroy(plan)
        del Ld
        torch.cuda.empty_cache()
        return e0.elapsed_time(e1) / args.steps, st

    d0 = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, n_spin=spec.n_spin, l_layout=layout, prec=pcode)
    nblk = 1 if spec.n_spin == 1 else 3
    full = [torch.empty(dm.dmet_emb_eri_bytes(d0, b) // 8, dtype=torch.float64, device="cuda") for b in range(nblk)]
    ms_full, st_full = one(None, full)
    total = [torch.zeros_like(t) for t in full]
    part = [torch.empty_like(t) for t in full]
    shard_ms, sts = [], []
    for r in ranges:
        ms, st = one(r, part)
        shard_ms.append(ms)
        sts.append(st)
        for t, x in zip(total, part):
            t += x
    diff = max(float(torch.linalg.norm(t - f) / torch.linalg.norm(f)) for t, f in zip(total, full))
    line = {"metric": METRIC, "workload": f"{args.workload}: q-shard split emulated shard by shard on one GPU",
            "shards": nshard, "q_ranges": ranges, "dtype": args.prec, "unsharded_ms": ms_full,
            "shard_ms": shard_ms, "sum_of_shards_ms": sum(shard_ms),
            "balance_max_over_mean": max(shard_ms) / (sum(shard_ms) / nshard),
            "slowest_shard_ms": max(shard_ms),
            "reduce_bytes_per_rank": int(sum(t.numel() * 8 for t in full)),
            "partial_sum_vs_unsharded_rel_fro": diff, "all_ok": st_full == 0 and all(x == 0 for x in sts),
            "note": "no multi-GPU time is claimed: the N-GPU step would be the slowest shard plus an FP64 "
                    "sum-reduce of reduce_bytes_per_rank over NCCL, neither measured together here"}
    print(json.dumps(line), flush=True)
    return 0


def _class_stats(dm, plan, name):
    for i in range(dm.dmet_emb_profile_count()):
        k = dm.dmet_emb_profile_read(plan, i)
        if k["name"] == name:
            return k
    return None


def run_rows_f(args):
    """The FP64 rows beside the hot path, each timed with CUDA events and checked against the oracle:
    density-fitted J/K straight from the factors L^q (h-BN-shaped, the L^q of dmet_emb_transform_3idx),
    and the FFTDF embedded ERI of Appendix B (a 2x2x2 mesh on a 12^3 cell grid)."""
    import torch
    import oracle
    import oracle.fftdf as of
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    libbuild.build()
    stream = torch.cuda.current_stream()
    f_peak = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
    reps = max(args.steps, 1)
    out = {"metric": METRIC, "workload": "rows_f (density-fitted J/K at the h-BN size; FFTDF on a 2x2x2 mesh)",
           "dtype": "f64"}
    # J/K: h-BN-shaped L^q (Nk 36, n_aux 220, n 104), restricted, real orbitals
    spec = synth.CONFIGS["hbn_6x6x1"]
    L, (C,), _ = synth.make_problem(spec)
    n, nk = spec.n_emb, spec.nk
    d = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n)
    Lq = torch.empty((nk, spec.n_aux, n, n), dtype=torch.complex128, device="cuda")
    gam = torch.from_numpy(synth.embedding_density(n, spec.seed).astype(np.complex128)).cuda()
    J = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(J)
    plan = dm.dmet_emb_plan(d, stream=stream.cuda_stream, workspace_limit=16 << 30)
    try:
        dm.dmet_emb_transform_3idx(plan, 0, torch.from_numpy(L).cuda(), [torch.from_numpy(C).cuda()], 0, nk, [Lq])
        for _ in range(args.warmup):
            dm.dmet_emb_jk_df(plan, Lq, gam, J, K)
        dm.dmet_emb_profile(plan, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            dm.dmet_emb_jk_df(plan, Lq, gam, J, K)
        e1.record(stream)
        torch.cuda.synchronize()
        ks = _class_stats(dm, plan, "jk_density_fitted")
        st = dm.dmet_emb_status(plan, 0)[0]
    finally:
        dm.dmet_emb_destroy(plan)
    ms = e0.elapsed_time(e1) / reps
    # the oracle's J and K from the same factors (the factors themselves are checked by the parity tests)
    Jr, Kr = oracle.coulomb_exchange_df(Lq.cpu().numpy(), gam.cpu().numpy(), spec.mesh)
    scale = float(np.abs(Jr).max())
    tf = ks["flops"] / reps / (ms / 1e3) / 1e12
    out["jk_df"] = {"config": {"mesh": list(spec.mesh), "n_aux": spec.n_aux, "n_emb": n}, "ms_per_call": ms,
                    "launches_per_call": ks["launches"] // reps, "status": st,
                    "roofline": {"bound": "alu", "achieved": tf, "peak": f_peak, "unit": "TFLOP/s", "frac": tf / f_peak,
                                 "flops_counted": "FP64 flops of the batched complex GEMMs (L^q gamma L^-q) and traces",
                                 "peak_source": "derived FP64 peak (152 SMs x 2 FMA/clk x 2 x 2070 MHz)"},
                    "max_abs_err_over_max_J": {"J": float(np.abs(J.cpu().numpy() - Jr).max()) / scale,
                                               "K": float(np.abs(K.cpu().numpy() - Kr).max()) / scale}}
    del Lq
    torch.cuda.empty_cache()
    # FFTDF: Algorithm 2 on a 2x2x2 mesh, 8 AOs per cell, 12^3 grid points, 16 embedding orbitals
    gspec = synth.GridSpec((2, 2, 2), 8, (12, 12, 12), n_emb=16, seed=5)
    rho = synth.pair_densities_k(gspec)
    Cg = synth.bloch_orbitals(synth.grid_orbitals(gspec), gspec.mesh)
    ng = int(np.prod(gspec.grid))
    d = dm.make_desc(gspec.mesh, gspec.n_ao, ng, gspec.n_emb, eri_pack=dm.binding.DMET_PACK_FULL)
    rd = torch.from_numpy(np.ascontiguousarray(rho.transpose(0, 1, 4, 2, 3))).cuda()
    Cd = [torch.from_numpy(Cg).cuda()]
    eo = torch.empty(dm.dmet_emb_eri_bytes(d, 0) // 16, dtype=torch.complex128, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=stream.cuda_stream, workspace_limit=16 << 30)
    try:
        for _ in range(args.warmup):
            dm.dmet_emb_eri_fftdf(plan, rd, Cd, gspec.grid, gspec.lattice, [eo])
        dm.dmet_emb_profile(plan, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            dm.dmet_emb_eri_fftdf(plan, rd, Cd, gspec.grid, gspec.lattice, [eo])
        e1.record(stream)
        torch.cuda.synchronize()
        ks = _class_stats(dm, plan, "fftdf_grid")
        kern_f = kernel_table([dm.dmet_emb_profile_read(plan, k) for k in range(dm.dmet_emb_profile_count())])
        st = dm.dmet_emb_status(plan, 0)[0]
    finally:
        dm.dmet_emb_destroy(plan)
    ms = e0.elapsed_time(e1) / reps
    ref = of.embedded_eri_fftdf(rho, Cg, gspec.mesh, gspec.lattice, gspec.grid).ravel()
    got = eo.cpu().numpy()
    # the roofline of the FFTDF steps themselves (the phases, the per-axis DFT GEMMs, the kernel and the
    # contraction over the grid) over their own event time; the half transforms before them are Algorithm 1's
    tf = ks["flops"] / (ks["ms"] / 1e3) / 1e12 if ks["ms"] > 0 else 0.0
    out["fftdf"] = {"config": {"mesh": list(gspec.mesh), "n_ao": gspec.n_ao, "grid": list(gspec.grid),
                               "n_emb": gspec.n_emb}, "ms_per_call": ms,
                    "launches_per_call": sum(k["launches"] for k in kern_f.values()) // reps,
                    "status": st, "kernels": kern_f,
                    "roofline": {"bound": "alu", "kernel": "fftdf_grid", "achieved": tf, "peak": f_peak,
                                 "unit": "TFLOP/s", "frac": tf / f_peak,
                                 "flops_counted": "FP64 flops of the per-axis DFT GEMMs, the phases and the "
                                                  "contraction over the grid",
                                 "peak_source": "derived FP64 peak (152 SMs x 2 FMA/clk x 2 x 2070 MHz)"},
                    "max_abs_err_over_max": float(np.abs(got - ref).max() / np.abs(ref).max())}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="bf16x3", choices=sorted(PREC_CODES),
                    help="path of the headline number")
    ap.add_argument("--precs", default="fp64",
                    help="comma-separated paths measured alongside the headline (errors included)")
    ap.add_argument("--only", action="store_true", help="measure the headline path only")
    ap.add_argument("--l-layout", default="auto", choices=["auto", "full", "reduced"],
                    help="auto: reduced when the full L would exceed 32 GB")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="timed steps of the FP64 path (-1: 3, or 0 when one FP64 call would exceed a minute)")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="timed end-to-end steps (-1: 3, or 2 above 100 GB)")
    ap.add_argument("--e2e-qblock", type=int, default=1,
                    help="q-block cap (DMET_QBLOCK) of the end-to-end plan; 0 = the plan's own choice")
    ap.add_argument("--check-orbitals", type=int, default=-1,
                    help="orbitals per spin of the seeded subset on which the oracle checks every result "
                         "(-1: 48, or 24 when L exceeds 100 GB, where the oracle streams every aux function's "
                         "L and its time grows with the subset)")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle check and the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="the default workload's line without its batch48 summary")
    ap.add_argument("--emulate-shards", type=int, default=0,
                    help="run the q-shard split of the workload over this many shards one after another on this "
                         "GPU (each shard timed alone; the shards' FP64 partial sum checked against one call)")
    ap.add_argument("--multi", default="weak", choices=["weak", "qshard"],
                    help="N > 1: weak = one problem per rank (no exchange); qshard = one problem split into q "
                         "shards over the ranks, with an FP64 sum of the partial ERIs (strong scaling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)
    if args.emulate_shards > 1:
        return run_shard_emulation(args)
    if args.workload == "batch48":
        return run_batch(args)
    if args.workload == "batch48_stated":
        return run_batch_stated(args)
    if args.workload == "hbn_6x6x1_complex":
        return run_complex(args)
    if args.workload == "rows_f":
        return run_rows_f(args)

    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild
    from synth import gpu as sgpu

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()

    base = synth.CONFIGS[args.workload]
    qshard = world > 1 and args.multi == "qshard"
    # Weak scaling: every rank transforms its own problem (a different seed); no data exchange.
    # q shards: every rank takes its share of the contracted q of the same problem (strong scaling).
    spec = base if qshard else rank_spec(base, rank)
    n_list = [spec.n_emb] * spec.n_spin
    q_range = shard_ranges(spec.mesh, spec.n_ao, n_list, world)[rank] if qshard else None
    fl_total = useful_flops(spec, n_list)[0]
    full_L_bytes = spec.nk ** 2 * spec.n_aux * spec.n_ao ** 2 * 16
    reduced = args.l_layout == "reduced" or (args.l_layout == "auto" and full_L_bytes > (32 << 30))
    layout = dm.binding.DMET_L_REDUCED if reduced else dm.binding.DMET_L_FULL
    big = full_L_bytes > (32 << 30)

    # Inputs: C on the host (QR over the supercell), L drawn on the device by the seeded generator.
    _, Cs, _ = synth.make_problem(spec, with_L=False)
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    desc_kw = dict(n_spin=spec.n_spin, l_layout=layout, q_range=q_range)
    probe = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, **desc_kw)
    if reduced:
        pairs = dm.dmet_emb_l_pairs(probe)   # with a q shard, the shard's blocks only
    else:
        pairs = np.arange(spec.nk * spec.nk)
    t0 = time.perf_counter()
    holder = {"Ld": sgpu.make_L_pairs_device(torch, spec, pairs)}
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    L_bytes = holder["Ld"].numel() * 16

    n_check = args.check_orbitals if args.check_orbitals > 0 else (24 if L_bytes > (100 << 30) else 48)
    S = subset_orbitals(spec, n_check)
    positions = block_positions(spec, S)
    nblk = len(positions)

    extra = [] if args.only else [p for p in args.precs.split(",") if p and p != args.prec]
    for p in extra:
        if p not in PREC_CODES:
            raise SystemExit(f"unknown precision {p}")
    precs = [args.prec] + extra
    res, subs = {}, {}
    for prec in precs:
        pcode = PREC_CODES[prec]
        desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, prec=pcode, **desc_kw)
        if prec == "fp64":
            steps = args.fp64_steps if args.fp64_steps >= 0 else (0 if big else 3)
            if steps == 0:
                res[prec] = {"skipped": "one FP64 call on this workload takes minutes (the FP64 pipe runs at "
                                        "1/64 of the FP32 rate); measured on the smaller workloads"}
                continue
        else:
            steps = args.steps
        outs = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64, device="cuda")
                for b in range(nblk)]
        free, _ = torch.cuda.mem_get_info()
        ws_limit = max(1 << 30, free - (4 << 30))
        r = measure(dm, torch, spec, desc, holder["Ld"], Cd, outs, steps, args, dist, world, local, ws_limit,
                    autotune=(prec != "fp64" and not args.no_autotune and not big), qshard=qshard)
        subs[prec] = gather_subsets(torch, outs, positions)
        if prec == args.prec and spec.n_spin == 1:
            r["embedding_fock"], r["dmet_bath"] = measure_fock_and_bath(dm, torch, spec, Cd, outs[0])
        res[prec] = r
        del outs
        torch.cuda.empty_cache()
    head = res[args.prec]

    e2e = None
    if qshard and not args.no_e2e:
        e2e = {"skipped": "the q-shard mode times resident inputs only"}
    elif not args.no_e2e:
        need = L_bytes + sum(dm.dmet_emb_eri_bytes(probe, b) for b in range(nblk))
        avail = host_available_bytes()
        if avail and need * 1.25 > avail:
            e2e = {"skipped": f"host memory: {need / 1e9:.0f} GB of pinned buffers wanted, {avail / 1e9:.0f} GB "
                              f"available"}
        else:
            args.e2e_steps = args.e2e_steps if args.e2e_steps > 0 else (2 if L_bytes > 100e9 else 3)
            desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, prec=PREC_CODES[args.prec], **desc_kw)
            # the device L is released once its host copy exists; the plan's staging buffers then take
            # its place (L and the output blocks), so the workspace gets what is free now less the outputs
            free, _ = torch.cuda.mem_get_info()
            out_b = sum(dm.dmet_emb_eri_bytes(desc, b) for b in range(nblk))
            e2e, e2e_sub = measure_e2e(dm, torch, desc, holder, Cs, positions, fl_total, world, args,
                                       ws_limit=max(1 << 30, free - out_b - (8 << 30)))
            e2e["matches_device_result"] = bool(all(np.array_equal(a, b) for a, b in zip(e2e_sub, subs[args.prec])))
    holder["Ld"] = None
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": head["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": head["steps"],
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "strong" if qshard else "weak",
        "vs_baseline": None, "dtype": PREC_DTYPE[args.prec], "data": "synthetic",
        "config": {**workload_config(spec, args.prec, "reduced" if reduced else "full"),
                   "problems_per_step": 1 if qshard else world,
                   "parallelism": f"q shards over {world} GPUs, FP64 sum of the partial ERIs" if qshard else
                   (f"one problem per GPU ({world})" if world > 1 else "1 GPU"),
                   "l2": f"inputs larger than L2 (L = {L_bytes / 1e9:.2f} GB)"},
        "ms_per_problem": head["ms_per_step"],
        "useful_tflop_per_problem": head["useful_tflop_per_problem"],
        "useful_split": head["useful_split"],
        "roofline": head["roofline"],
        "kernels": head["kernels"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "e2e": e2e,
        "device_checks": head["device_checks"],
        "tile_widths": head.get("tile_widths"),
        "input_generation_s": gen_s,
    }
    if "embedding_fock" in head:
        line["embedding_fock"], line["dmet_bath"] = head["embedding_fock"], head["dmet_bath"]
    for p in precs[1:]:
        r = res[p]
        if "skipped" in r:
            line[p] = r
            continue
        line[p] = {k: r[k] for k in ("value", "ms_per_step", "roofline", "kernels", "gpu_launches", "clocks")}
        line[p]["dtype"] = PREC_DTYPE[p]
    if "value" in res.get("fp64", {}):
        line["speedup_over_fp64"] = {p: res["fp64"]["ms_per_step"] / res[p]["ms_per_step"]
                                     for p in res if p != "fp64" and "value" in res[p]}

    if rank == 0 and not args.no_check:
        # The oracle on the seeded orbital subsets (every aux function, streamed): the error of each GPU
        # result per spin block, and the oracle's own rate on the first blocks as the CPU baseline.
        # blocks of aux functions of about 24 GB of L (larger blocks: larger GEMMs in the oracle)
        pb = max(1, min(spec.n_aux, (24 << 30) // (spec.nk ** 2 * spec.n_ao ** 2 * 16)))
        refs, base, info = oracle_check(torch, spec, Cs, S, pb)
        names = {(0, 0): "aa" if spec.n_spin == 2 else "s8", (0, 1): "ab", (1, 1): "bb"}
        errs_all = {p: {names[k]: error_stats(subs[p][b], refs[b]) for b, k in enumerate(block_spins(spec))}
                    for p in subs}
        line["cpu_baseline"] = base
        line["error_vs_fp64_oracle"] = {"sample": f"all (ij|kl) of every spin block on seeded {len(S[0])}-orbital "
                                                  f"subsets per spin", **errs_all, "oracle": info}
    if rank == 0 and world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_batch:
        # the batched workload (48 uneven problems, grouped launches against the FP64 path) rides along
        # with the default line, so that every default run also records it
        try:
            b = batch_line(argparse.Namespace(**{**vars(args), "steps": 3, "warmup": 3, "fp64_steps": 1}),
                           arms=("bf16x3", "fp64"))
            keep = ("problems_per_s", "ms_per_batch", "useful_tflops", "p50_ms", "p99_ms", "latency",
                    "grouped_launches", "gpu_launches_per_batch", "all_ok", "steps", "max_rel_fro_vs_oracle")
            line["batch48"] = {"workload": b["workload"], **{a: {k: b[a][k] for k in keep if k in b[a]}
                                                             for a in ("bf16x3", "fp64")},
                               "speedup_bf16x3_over_fp64": b.get("speedup_bf16x3_over_fp64")}
        except Exception as e:  # the headline line is printed whatever happens here
            line["batch48"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
