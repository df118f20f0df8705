"""Benchmark of the embedded-ERI transformation (Algorithm 1 of arXiv 1909.08596, section 2.1).

One step = one call of dmet_emb_eri on one embedding problem: orbital and symmetry checks,
the k-AO -> k-EO half transforms of every needed (k1, k1+q) pair, the Fourier sum to the
reference cell, the contraction over the aux index and the sum over q into the 8-fold
packed ERI. Inputs are synthetic (seeded) with the h-BN-shaped sizes of section 2.2
(6x6x1 mesh, 26 AOs and 220 aux functions per cell, 104 embedding orbitals).

Prints one JSON line. `value` is useful TFLOP/s (the symmetry-reduced algorithmic flop
count of the work the library does) with inputs resident in HBM; `e2e` is the same metric
through the C ABI with host buffers (copies inside the timed region).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--workload NAME]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hbn_6x6x1")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)

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
    spec = synth.spec_with(base, seed=base.seed + 17 * rank)
    L, Cs, _ = synth.make_problem(spec)
    n_list = [spec.n_emb] * spec.n_spin
    fl_total, fl_t, fl_c = useful_flops(spec, n_list)

    stream = torch.cuda.current_stream()
    desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, n_list, n_spin=spec.n_spin)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    nblk = 1 if spec.n_spin == 1 else 3
    outs = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64, device="cuda") for b in range(nblk)]
    plan = dm.dmet_emb_plan(desc, stream=stream.cuda_stream)

    def step():
        dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])

    for _ in range(args.warmup):
        step()
    st, stats = dm.dmet_emb_status(plan, 0)
    if st != dm.binding.DMET_OK:
        raise RuntimeError(f"device status {st}: {dm.dmet_emb_last_error()} {stats}")

    # Timed region: K steps, CUDA events on the launching stream, barrier + sync both sides.
    dm.dmet_emb_profile(plan, True)
    launches0 = dm.dmet_emb_launch_count(plan)
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
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
    if dist:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = world * fl_total * args.steps / (ms_total / 1e3) / 1e12

    # Dominant kernel: the class with the most device time in the timed region.
    top = max(kstats, key=lambda k: k["ms"])
    peak_fp64 = SMS * DFMA_PER_SM_CLK * 2 * 2070e6 / 1e12
    achieved = top["flops"] / (top["ms"] / 1e3) / 1e12 if top["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel": top["name"], "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
                "frac": achieved / peak_fp64, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (FP64 runs on the CUDA cores)",
                "avg_launch_ms": top["ms"] / max(top["launches"], 1)}
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["ms"], 3),
                           "share": round(k["ms"] / max(sum(x["ms"] for x in kstats), 1e-9), 4)}
               for k in kstats if k["launches"]}

    # End to end through the C ABI with host buffers: H2D of L and C, D2H of the ERI.
    Lh = torch.from_numpy(L).pin_memory()
    Ch = [torch.from_numpy(c).pin_memory() for c in Cs]
    Oh = [torch.empty(o.numel(), dtype=torch.float64).pin_memory() for o in outs]
    dm.dmet_emb_eri(plan, [Lh], [Ch], [Oh])  # warm the staging buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        dm.dmet_emb_eri(plan, [Lh], [Ch], [Oh])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    h2d = Lh.numel() * 16 + sum(c.numel() * 16 for c in Ch)
    d2h = sum(o.numel() * 8 for o in Oh)
    st, stats = dm.dmet_emb_status(plan, 0)
    same = all(torch.equal(o.cpu(), h) for o, h in zip(outs, Oh))

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec.name, "mesh": list(spec.mesh), "n_ao": spec.n_ao, "n_aux": spec.n_aux,
                   "n_emb": spec.n_emb, "n_spin": spec.n_spin, "prec": "fp64", "pack": "s8",
                   "problems_per_step": world, "l2": f"inputs larger than L2 (L = {L.nbytes / 1e9:.2f} GB)"},
        "ms_per_problem": ms_step,
        "useful_tflop_per_problem": fl_total / 1e12,
        "useful_split": {"transform": fl_t / 1e12, "contraction": fl_c / 1e12},
        "roofline": roofline,
        "kernels": kernels,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": world * fl_total / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3, "matches_device_result": bool(same)},
        "device_checks": {"status": int(st), "orthonormality": stats[0], "realness": stats[1],
                          "hermiticity_L": stats[2], "time_reversal_L": stats[3]},
    }

    if rank == 0 and not args.no_cpu_baseline:
        # CPU baseline: the oracle as it stands on a bounded sample (orbital subset) of this
        # workload, also giving the error of the GPU result on that subset.
        dt, fl_s, S, eri_s = oracle_sample(spec, L, Cs[0], 32)
        got = outs[0].cpu().numpy()
        i, j, k, l = np.meshgrid(*([np.arange(len(S))] * 4), indexing="ij")
        ii, jj, kk, ll = S[i.ravel()], S[j.ravel()], S[k.ravel()], S[l.ravel()]
        I, J = np.maximum(ii, jj), np.minimum(ii, jj)
        K_, L_ = np.maximum(kk, ll), np.minimum(kk, ll)
        a, b = I * (I + 1) // 2 + J, K_ * (K_ + 1) // 2 + L_
        P, Q = np.maximum(a, b), np.minimum(a, b)
        g = got[P * (P + 1) // 2 + Q]
        ref = eri_s.real.ravel()
        line["cpu_baseline"] = {"value": fl_s / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"Algorithm 1 (all q, all k1, dense contraction) on 32 of {spec.n_emb} "
                                          f"embedding orbitals; {dt:.1f} s; useful flops of that sub-problem"}
        line["error_vs_fp64_oracle"] = {
            "rel_fro": float(np.linalg.norm(g - ref) / np.linalg.norm(ref)),
            "max_abs": float(np.abs(g - ref).max()), "max_abs_over_max": float(np.abs(g - ref).max() / np.abs(ref).max()),
            "rms": float(np.sqrt(np.mean((g - ref) ** 2))), "sample": "all (ij|kl) on the 32-orbital subset"}
    dm.dmet_emb_destroy(plan)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
