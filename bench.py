"""Benchmark of the embedded-ERI transformation (Algorithm 1 of arXiv 1909.08596, section 2.1).

One step = one call of dmet_emb_eri on one embedding problem: orbital and symmetry checks,
the k-AO -> k-EO half transforms of every needed (k1, k1+q) pair, the Fourier sum to the
reference cell, the contraction over the aux index and the sum over q into the 8-fold
packed ERI. Inputs are synthetic (seeded) with the h-BN-shaped sizes of section 2.2
(6x6x1 mesh, 26 AOs and 220 aux functions per cell, 104 embedding orbitals).

Prints one JSON line. `value` is useful TFLOP/s (the symmetry-reduced algorithmic flop
count of the work the library does) with inputs resident in HBM; `e2e` is the same metric
through the C ABI with host buffers (copies inside the timed region). The headline path is
the split-BF16 tensor-core path; the plain FP64 path is measured in the same run and
reported under "fp64", and both are compared with the FP64 oracle on an orbital subset.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--workload NAME]
                    [--prec bf16x3|fp64] [--only]
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
SMS = 152
DFMA_PER_SM_CLK = 2  # FP64 FMA lanes per SM per clock on GB300 (1.25 TFLOP/s nominal at 2.07 GHz)
ORACLE_SAMPLE_ORBITALS = 24
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the tensor kernels, averaged over the launches of
# one call, from a one-pass ncu capture of the full h-BN bench command (profiles/launches_bf16x3_hbn_6x6x1.txt
# gives the command and the figures); (workload, path, kernel class) -> bytes. Valid only for the kernels as
# they were at that capture.
TRAFFIC = {
    ("hbn_6x6x1", "bf16x3", "tc_half_transform_1"): 1.424e9,
    ("hbn_6x6x1", "bf16x3", "tc_half_transform_2"): 1.154e9,
    ("hbn_6x6x1", "bf16x3", "tc_contract"): 1.273e9,
}


def useful_flops(spec, n_list, desc_sym=1):
    """Algorithmic flops of one problem with the symmetry reductions the library applies.

    Transform (per spin, per computed pair): 8 n_aux (n_ao^2 n + n_ao n^2) (a complex MAC is
    8 flops); contraction: npair (npair+1) K per same-spin block, 2 npair_a npair_b K for
    alpha-beta, K = n_aux * (1 + [q != -q]) summed over the contracted q."""
    import paper_1909_08596_gb300 as dm
    d = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, n_spin=len(n_list), sym=desc_sym)
    s = dm.dmet_emb_schedule(d)
    nao, naux = spec.n_ao, spec.n_aux
    fl_t = 0.0
    K = 0
    for q in range(spec.nk):
        w = s["q_weight"][q]
        if not w:
            continue
        K += naux * (1 if w == 1 else 2)
        for n in n_list:
            fl_t += s["n_rep"][q] * 8.0 * naux * (nao * nao * n + nao * n * n)
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
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


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


def job_tflops(world, flops_per_problem, steps, ms_total):
    """Whole-job throughput: every rank's problems over the slowest rank's time."""
    return world * flops_per_problem * steps / (ms_total / 1e3) / 1e12


def oracle_sample(spec, L, C, n_sub, seed=0):
    """Runs the CPU oracle (Algorithm 1 as written: every q, every k1, dense contraction) on a
    seeded subset of n_sub embedding orbitals; returns (seconds, useful flops, orbital subset,
    ERI on the subset). Orbital-column subsets of the ERI are exact (same arithmetic per entry)."""
    import oracle
    rng = np.random.default_rng(seed)
    S = np.sort(rng.choice(C.shape[2], n_sub, replace=False))
    t0 = time.perf_counter()
    eri = oracle.embedded_eri(L, np.ascontiguousarray(C[:, :, S]), spec.mesh)
    dt = time.perf_counter() - t0
    return dt, useful_flops(spec, [n_sub])[0], S, eri


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    spec = synth.CONFIGS[args.workload]
    L, (C,), _ = synth.make_problem(spec)
    times, fl = [], 0.0
    for it in range(args.warmup + args.steps):
        dt, fl, _, _ = oracle_sample(spec, L, C, ORACLE_SAMPLE_ORBITALS, seed=it)
        if it >= args.warmup:
            times.append(dt)
    sec = float(np.mean(times))
    value = fl / sec / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec.name, "mesh": list(spec.mesh), "n_ao": spec.n_ao, "n_aux": spec.n_aux,
                   "n_emb": spec.n_emb, "sample_orbitals": ORACLE_SAMPLE_ORBITALS},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"Algorithm 1 (all q, all k1, dense contraction) on {ORACLE_SAMPLE_ORBITALS} "
                                   f"of {spec.n_emb} embedding orbitals per step; useful flops of that sub-problem"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def s8_positions(S):
    """Packed 8-fold indices of every (ij|kl) with i, j, k, l in the orbital subset S."""
    i, j, k, l = np.meshgrid(*([np.arange(len(S))] * 4), indexing="ij")
    ii, jj, kk, ll = S[i.ravel()], S[j.ravel()], S[k.ravel()], S[l.ravel()]
    I, J = np.maximum(ii, jj), np.minimum(ii, jj)
    K_, L_ = np.maximum(kk, ll), np.minimum(kk, ll)
    a, b = I * (I + 1) // 2 + J, K_ * (K_ + 1) // 2 + L_
    P, Q = np.maximum(a, b), np.minimum(a, b)
    return P * (P + 1) // 2 + Q


def measure(dm, torch, spec, L, Cs, Ld, Cd, prec, args, dist, world, local):
    """Times args.steps calls of dmet_emb_eri on resident inputs, then the end-to-end form."""
    n_list = [spec.n_emb] * spec.n_spin
    fl_total, fl_t, fl_c = useful_flops(spec, n_list)
    stream = torch.cuda.current_stream()
    pcode = dm.binding.DMET_PREC_FP64 if prec == "fp64" else dm.binding.DMET_PREC_BF16X3
    desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, n_spin=spec.n_spin, prec=pcode)
    nblk = 1 if spec.n_spin == 1 else 3
    outs = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64, device="cuda") for b in range(nblk)]
    plan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream)
    tile_widths = None
    if prec != "fp64" and not args.no_autotune:
        # Tile widths of the transform GEMMs chosen by timing (outside the timed region).
        dm.dmet_emb_autotune(plan, [Ld], [Cd], [outs])
        tile_widths = dm.dmet_emb_tile_widths(plan, 0)

    def step():
        dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])

    for _ in range(args.warmup):
        step()
    st, stats = dm.dmet_emb_status(plan, 0)
    if st != dm.binding.DMET_OK:
        raise RuntimeError(f"device status {st}: {dm.dmet_emb_last_error()} {stats}")
    steps = args.steps if prec != "fp64" else min(args.steps, args.fp64_steps)
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
    ms_total = max_over_ranks(dist, ms_total, "cuda")
    ms_step = ms_total / steps
    value = job_tflops(world, fl_total, steps, ms_total)

    peaks, peak_src = measured_peaks()
    top = max(kstats, key=lambda k: k["ms"])
    avg_ms = top["ms"] / max(top["launches"], 1)
    if prec == "fp64":
        peak = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
        achieved = top["flops"] / (top["ms"] / 1e3) / 1e12 if top["ms"] > 0 else 0.0
        roof = {"bound": "alu", "kernel": top["name"], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": TRAFFIC.get((spec.name, prec, top["name"])),
                "flops_counted": "algorithmic FP64 flops",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (FP64 runs on the CUDA cores)",
                "avg_launch_ms": avg_ms}
    else:
        # A tensor kernel's roofline is whichever of its two floors is higher: executed tensor
        # flops at the measured bf16 peak, or its algorithmic bytes at the measured HBM copy rate.
        peak_t, peak_b = peaks["bf16_tflops"], peaks["hbm_gbs"]
        secs = top["ms"] / 1e3 / max(top["launches"], 1)
        fl_l = top["exec_flops"] / max(top["launches"], 1)
        by_l = top["bytes"] / max(top["launches"], 1)
        t_tensor, t_hbm = fl_l / (peak_t * 1e12), by_l / (peak_b * 1e9)
        tensor = {"achieved": fl_l / secs / 1e12 if secs > 0 else 0.0, "peak": peak_t, "unit": "TFLOP/s"}
        hbm = {"achieved": by_l / secs / 1e9 if secs > 0 else 0.0, "peak": peak_b, "unit": "GB/s"}
        for d in (tensor, hbm):
            d["frac"] = d["achieved"] / d["peak"]
        main, other = (hbm, tensor) if t_hbm > t_tensor else (tensor, hbm)
        roof = {"bound": "hbm" if main is hbm else "tensor", "kernel": top["name"], **main,
                "traffic": TRAFFIC.get((spec.name, prec, top["name"])),
                "other_bound": {"bound": "tensor" if main is hbm else "hbm", **other},
                "flops_counted": "executed BF16 tensor flops (6 slice products per useful multiply-add, whole tiles)",
                "bytes_counted": "algorithmic bytes per launch: operands read once, result written once",
                "useful_achieved_tflops": top["flops"] / (top["ms"] / 1e3) / 1e12 if top["ms"] > 0 else 0.0,
                "peak_source": f"{peak_src} bf16_tflops (burst; sustained {peaks.get('bf16_tflops_sustained')}) "
                               f"and hbm_gbs",
                "avg_launch_ms": avg_ms}
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
        kernels[k["name"]] = e

    # The embedding one-particle Hamiltonian from this ERI (dmet_emb_fock, FP64 kernels): timed on
    # its own, after the ERI, with a synthetic mean-field Fock matrix and embedding density.
    fock = None
    if spec.n_spin == 1:
        Fk = torch.from_numpy(synth.fock_k(synth.real_space_fock(spec), spec.mesh)).cuda()
        gam = torch.from_numpy(synth.embedding_density(spec.n_emb, spec.seed)).cuda()
        fo = torch.empty((spec.n_emb, spec.n_emb), dtype=torch.float64, device="cuda")
        for _ in range(3):
            dm.dmet_emb_fock(plan, Fk, Cd[0], outs[0], gam, fo)
        dm.dmet_emb_profile(plan, True)
        reps = 10
        ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ef0.record(stream)
        for _ in range(reps):
            dm.dmet_emb_fock(plan, Fk, Cd[0], outs[0], gam, fo)
        ef1.record(stream)
        torch.cuda.synchronize()
        fk = [k for k in (dm.dmet_emb_profile_read(plan, i) for i in range(dm.dmet_emb_profile_count()))
              if k["name"] == "embedding_fock"][0]
        dm.dmet_emb_profile(plan, False)
        f_ms = ef0.elapsed_time(ef1) / reps
        f_peak = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
        f_tf = fk["flops"] / reps / (f_ms / 1e3) / 1e12
        fock = {"ms": f_ms, "launches_per_call": fk["launches"] // reps,
                "roofline": {"bound": "alu", "achieved": f_tf, "peak": f_peak, "unit": "TFLOP/s", "frac": f_tf / f_peak,
                             "flops_counted": "FP64 flops the kernels execute (transform GEMMs; 2 n^2 exchange and "
                                              "n(n+1)/2 Coulomb multiply-adds per ERI pair row)",
                             "peak_source": "derived FP64 peak (152 SMs x 2 FMA/clk x 2 x 2070 MHz)"}}

    # The DMET bath that produces such orbitals (dmet_emb_bath, FP64 kernels): the same cell and
    # mesh, its n_AO LOs as the impurity and 8 of them as the valence columns of the SVD (the
    # valence shell of a two-atom s/p cell), from a synthetic gapped mean field.
    bath = None
    if spec.n_spin == 1 and spec.nk > 1:
        n_val = min(8, spec.n_ao)
        bspec = synth.spec_with(spec, n_emb=spec.n_ao + n_val)
        h = synth.mean_field_hamiltonian(bspec, spec.n_ao // 2)
        gk = torch.from_numpy(synth.mean_field_density(h, spec.mesh, spec.n_ao // 2)).cuda()
        Ulo = torch.from_numpy(synth.lo_rotation(bspec)).cuda()
        val = list(range(0, spec.n_ao, max(1, spec.n_ao // n_val)))[:n_val]
        Cb = torch.empty((spec.nk, spec.n_ao, bspec.n_emb), dtype=torch.complex128, device="cuda")
        binfo = torch.zeros(n_val + 5, dtype=torch.float64, device="cuda")
        bplan = dm.dmet_emb_plan(dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, bspec.n_emb), stream=stream.cuda_stream)
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

    # End to end through the C ABI with host buffers: H2D of L and C, D2H of the ERI. A plan of its
    # own, built with the q-block size capped (DMET_QBLOCK) so that L streams in small blocks.
    e2e = None
    if not args.no_e2e:
        Lh = torch.from_numpy(L).pin_memory()
        Ch = [torch.from_numpy(c).pin_memory() for c in Cs]
        Oh = [torch.empty(o.numel(), dtype=torch.float64).pin_memory() for o in outs]
        old_qb = os.environ.get("DMET_QBLOCK")
        if args.e2e_qblock > 0:
            os.environ["DMET_QBLOCK"] = str(args.e2e_qblock)
        try:
            eplan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream)
        finally:
            if old_qb is None:
                os.environ.pop("DMET_QBLOCK", None)
            else:
                os.environ["DMET_QBLOCK"] = old_qb
        try:
            outs_e = [torch.empty_like(o) for o in outs]
            if prec != "fp64" and not args.no_autotune:
                dm.dmet_emb_autotune(eplan, [Ld], [Cd], [outs_e])
            dm.dmet_emb_eri(eplan, [Ld], [Cd], [outs_e])  # the device result of this plan, for the check below
            dm.dmet_emb_eri(eplan, [Lh], [Ch], [Oh])
            torch.cuda.synchronize()
            e2e_steps = args.e2e_steps if prec != "fp64" else 1
            dm.dmet_emb_profile(eplan, False)  # clears the counters (no events are recorded)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                dm.dmet_emb_eri(eplan, [Lh], [Ch], [Oh])
            torch.cuda.synchronize()
            e2e_s = (time.perf_counter() - t0) / e2e_steps
            # bytes the library moved between host and device (it transfers only the L blocks its schedule reads)
            copy_b = sum(k["bytes"] for k in (dm.dmet_emb_profile_read(eplan, i)
                                              for i in range(dm.dmet_emb_profile_count()))
                         if k["name"] == "host_copy") / e2e_steps
        finally:
            dm.dmet_emb_destroy(eplan)
        d2h_b = int(sum(o.numel() * 8 for o in Oh))
        same = all(torch.equal(o.cpu(), h) for o, h in zip(outs_e, Oh))
        del outs_e
        e2e = {"value": world * fl_total / e2e_s / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(copy_b) - d2h_b, "d2h_bytes_per_step": d2h_b,
               "host_L_bytes": int(Lh.numel() * 16), "ms_per_step": e2e_s * 1e3,
               "qblock_cap": args.e2e_qblock, "matches_device_result": bool(same)}
    st, stats = dm.dmet_emb_status(plan, 0)
    dm.dmet_emb_destroy(plan)
    return {
        "value": value, "ms_per_step": ms_step, "useful_tflop_per_problem": fl_total / 1e12,
        "useful_split": {"transform": fl_t / 1e12, "contraction": fl_c / 1e12},
        "roofline": roof, "kernels": kernels, "gpu_launches": int(launches), "clocks": clk, "steps": steps,
        "tile_widths": tile_widths,
        "e2e": e2e,
        "device_checks": {"status": int(st), "orthonormality": stats[0], "realness": stats[1],
                          "hermiticity_L": stats[2], "time_reversal_L": stats[3]},
        "embedding_fock": fock,
        "dmet_bath": bath,
        "result": [o.cpu().numpy() for o in outs],
    }


def run_batch(args):
    """48 uneven problems in one plan (concurrent streams, CUDA-graph replay): problems/s and the
    p50/p99 per-problem device latency, FP64 and split-BF16."""
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
    for prec in ("bf16x3", "fp64"):
        pcode = dm.binding.DMET_PREC_FP64 if prec == "fp64" else dm.binding.DMET_PREC_BF16X3
        descs = [dm.make_desc(sp.mesh, sp.n_ao, sp.n_aux, sp.n_emb, n_spin=sp.n_spin, prec=pcode) for sp in specs]
        outs = [[torch.empty(dm.dmet_emb_eri_bytes(d, b) // 8, dtype=torch.float64, device="cuda")
                 for b in range(1 if d.n_spin == 1 else 3)] for d in descs]
        with torch.cuda.stream(stream):
            plan = dm.dmet_emb_plan(descs, stream=stream.cuda_stream, workspace_limit=64 << 30)
            # per-problem device latency from one profiled (non-graph) call
            dm.dmet_emb_profile(plan, True)
            dm.dmet_emb_eri(plan, Ls, Cds, outs)
            lat = sorted(dm.dmet_emb_problem_ms(plan, p) for p in range(len(specs)))
            dm.dmet_emb_profile(plan, False)
            dm.dmet_emb_graph(plan, True)
            for _ in range(args.warmup):
                dm.dmet_emb_eri(plan, Ls, Cds, outs)
            steps = args.steps if prec != "fp64" else min(args.steps, args.fp64_steps)
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
        out[prec] = {"problems_per_s": len(specs) / (ms / 1e3), "ms_per_batch": ms, "useful_tflops": fl / (ms / 1e3) / 1e12,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "gpu_launches": int(launches), "all_ok": all(x == 0 for x in st), "steps": steps}
        results[prec] = [[o.cpu().numpy() for o in row] for row in outs]
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
            "unit": "TFLOP/s", "problems": len(specs), **{p: out[p] for p in out},
            "speedup_bf16x3_over_fp64": out["fp64"]["ms_per_batch"] / out["bf16x3"]["ms_per_batch"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hbn_6x6x1")
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "fp64"],
                    help="path of the headline number; the other path is measured alongside unless --only")
    ap.add_argument("--only", action="store_true", help="measure the headline path only")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-qblock", type=int, default=1,
                    help="q-block cap (DMET_QBLOCK) of the end-to-end plan; 0 = the plan's own choice")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end measurement (it pins a host copy of L: for the largest workloads)")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch48":
        return run_batch(args)

    import torch
    import paper_1909_08596_gb300 as dm
    from paper_1909_08596_gb300 import build as libbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()

    base = synth.CONFIGS[args.workload]
    # Weak scaling: every rank transforms its own problem (a different seed); no data exchange.
    spec = rank_spec(base, rank)
    L, Cs, _ = synth.make_problem(spec)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]

    precs = [args.prec] + ([] if args.only else [p for p in ("bf16x3", "fp64") if p != args.prec])
    res = {p: measure(dm, torch, spec, L, Cs, Ld, Cd, p, args, dist, world, local) for p in precs}
    head = res[args.prec]

    line = {
        "metric": METRIC, "value": head["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": head["steps"],
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "bf16x3", "data": "synthetic",
        "config": {"workload": spec.name, "mesh": list(spec.mesh), "n_ao": spec.n_ao, "n_aux": spec.n_aux,
                   "n_emb": spec.n_emb, "n_spin": spec.n_spin, "prec": args.prec, "pack": "s8",
                   "problems_per_step": world, "l2": f"inputs larger than L2 (L = {L.nbytes / 1e9:.2f} GB)"},
        "ms_per_problem": head["ms_per_step"],
        "useful_tflop_per_problem": head["useful_tflop_per_problem"],
        "useful_split": head["useful_split"],
        "roofline": head["roofline"],
        "kernels": head["kernels"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "device_checks": head["device_checks"],
        "tile_widths": head.get("tile_widths"),
        "embedding_fock": head.get("embedding_fock"),
        "dmet_bath": head.get("dmet_bath"),
    }
    for p in precs[1:]:
        r = res[p]
        line[p] = {k: r[k] for k in ("value", "ms_per_step", "roofline", "kernels", "gpu_launches", "clocks", "e2e")}
        line[p]["dtype"] = "f64" if p == "fp64" else "bf16x3"
    if "fp64" in res and "bf16x3" in res:
        line["speedup_bf16x3_over_fp64"] = res["fp64"]["ms_per_step"] / res["bf16x3"]["ms_per_step"]

    if rank == 0 and not args.no_cpu_baseline:
        # CPU baseline: the oracle as it stands on a bounded sample (orbital subset) of this
        # workload, which also gives the error of each GPU result on that subset.
        dt, fl_s, S, eri_s = oracle_sample(spec, L, Cs[0], 32)
        pos = s8_positions(S)
        ref = eri_s.real.ravel()
        line["cpu_baseline"] = {"value": fl_s / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"Algorithm 1 (all q, all k1, dense contraction) on 32 of {spec.n_emb} "
                                          f"embedding orbitals; {dt:.1f} s; useful flops of that sub-problem"}
        errs = {}
        for p, r in res.items():
            g = r["result"][0][pos]
            errs[p] = {"rel_fro": float(np.linalg.norm(g - ref) / np.linalg.norm(ref)),
                       "max_abs": float(np.abs(g - ref).max()),
                       "max_abs_over_max": float(np.abs(g - ref).max() / np.abs(ref).max()),
                       "rms": float(np.sqrt(np.mean((g - ref) ** 2)))}
        line["error_vs_fp64_oracle"] = {"sample": "all (ij|kl) on a seeded 32-orbital subset", **errs}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
