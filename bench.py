"""Throughput benchmark of the fused-operator state-vector path on GB300.

Workload (one "step" = one pass of the whole hot path over one synthetic
circuit): QAOA on a seeded random 3-regular graph, N = 30 qubits, p = 8
rounds (H on every qubit, then 8 x (ZZ on 45 edges + RX on 30 qubits) = 630
gates), complex64 state of 8 GiB.  A step resets the state to |0...0>,
executes the fused plan (fused k-qubit blocks; FP32 CUDA cores, or split-TF32
tensor cores for k = 5, 6), reduces the norm in FP64, draws 1000 sampled
counts and evaluates <Z_a Z_b> on one edge.  The plan (cost-model training,
fusion, block products) is built once before the timed region, as the
paper's timer excludes plan construction.

Metric: gate-level amplitude-updates/s = (input gates x 2^N) / step time,
whole job (sum over ranks).  Multi-GPU runs are independent replicas (the
path is not sharded): weak scaling, no collective on the data path.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (one gate of the circuit per step at N = 28) on the host cores.

``--workload dm_ghz`` measures the density-matrix path instead: noisy GHZ on
n = 15 qubits (H, then CNOT(0 -> q) for q = 1..14, depolarising noise p = 0.01
after every gate: 30 channels), held as vec(rho) on 2n = 30 qubits; each
channel is lowered to its 2k-axis superoperator and the lowered circuit is
fused and executed like any other (one step: reset, execute, trace and
Tr(rho Z_0 Z_14)).  Its metric counts 4^n amplitude updates per channel.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "amplitude-updates/s"
UNIT = "amp-updates/s"

# DRAM bytes (read + write) per amplitude of one launch, from single ncu captures
# at N=28 (profiles/k_apply_tc6_n28.md: 4.241 GB; profiles/k_apply_fp32_k4_n28.md:
# 4.234 GB; profiles/k_apply_diag_n28.md: 4.234 GB; profiles/k_apply_prod_n28.md:
# 4.260 GB; profiles/k_apply_layer_n28.md: 4.265 GB (a regular pass); each /
# 2^28).  Traffic scales with the state size, so a launch at N moves this many
# bytes times 2^N.
DRAM_BYTES_PER_AMP = {"k_apply_tc": 4.234e9 / 2**28, "k_apply_fp32": 4.234e9 / 2**28,
                      "k_apply_diag": 4.234e9 / 2**28, "k_apply_prod": 4.260e9 / 2**28,
                      "k_apply_layer": 4.266e9 / 2**28}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; started
    before the warm-up so that it is running when the timed region begins, and
    read back for the samples stamped inside that region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Median SM clock, maximum clock and throttle reasons of the samples
        stamped in [t0, t1] (wall-clock seconds; all samples if none are)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append((ts, float(parts[2]), float(parts[3]),
                             [nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 is not None and r[0] is not None and t0 <= r[0] <= t1]
        use = inside or rows
        sm = [r[1] for r in use]
        mx = [r[2] for r in use]
        reasons = sorted({nm for r in use for nm in r[3]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm), "window": "timed region" if inside else "whole run"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_seconds(elapsed: float, ws: int, device=None) -> float:
    """Whole-job time of a replica run: the slowest rank's timed region (max
    over ranks, then a barrier); the replicas share no data, so this is the
    only collective."""
    if ws <= 1:
        return elapsed
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(units_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job time."""
    return ws * units_per_rank / seconds


def host_cpu():
    """The host's logical core count and CPU model (lscpu's model name, else
    /proc/cpuinfo, else the platform string)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"host_nproc": os.cpu_count(), "host_cpu": model or platform.processor() or platform.machine(),
            "host_arch": platform.machine()}


def run_reference(args):
    """The FP64 CPU oracle, unmodified, on a bounded sample of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    n_s = args.ref_qubits
    if args.workload == "dm_ghz":
        picks, _, what = _dm_oracle_picks(n_s // 2, args.dm_p)
        n_s = 2 * (n_s // 2)
        wl = f"dm_ghz{args.dm_n}"
    elif args.workload == "wide":
        n_s = min(n_s, 24)   # a k = 6 operator costs 64 complex products per amplitude on the host
        picks = W.wide_circuit(n_s, n_ops=2, widths=(5, 6), seed=args.seed)
        wl, what = f"wide{args.n}", "k=5 / k=6 Haar operator of the wide workload"
    elif args.workload == "fusion":
        picks = _fusion_picks(n_s, args.seed)
        wl, what = f"fusion{args.n}", "U(2) / U(4) gate of the fusion workload"
    else:
        ops, _ = W.qaoa_circuit(n=n_s, p=args.p, seed=args.seed)
        picks = [ops[0], ops[n_s]]   # alternate a one-qubit and a two-qubit gate of the circuit
        wl, what = f"qaoa{args.n}_p{args.p}", "H / ZZ gate of the QAOA circuit"
    psi = oracle.zero_state(n_s)
    times = []
    for i in range(args.warmup + args.steps):
        g = picks[i % 2]
        t0 = time.perf_counter()
        oracle.apply(psi, g.targets, g.matrix)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per_gate = statistics.mean(times)
    rate = (1 << n_s) / per_gate
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_gate * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl, "sample": f"one gate per step at N={n_s}"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"alternating {what} at N={n_s}, {args.steps} timed gates", **host_cpu()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _fusion_picks(n: int, seed: int):
    """A one-qubit and a two-qubit Haar gate of the fusion workload's layers."""
    ops, _ = W.fusion_circuit(n=n, layers=1, seed=seed, with_inverse=False)
    one = next(o for o in reversed(ops) if len(o.targets) == 1)
    two = next(o for o in reversed(ops) if len(o.targets) == 2)
    return [one, two]


class _LoweredOp:
    def __init__(self, targets, matrix):
        self.targets, self.matrix = tuple(targets), matrix


def _dm_oracle_picks(n_dm: int, p_dep: float):
    """Two channels of the noisy GHZ circuit (the first CNOT and its
    depolarising noise) lowered by the oracle to superoperators on vec(rho)
    of 2 n_dm qubits."""
    import oracle
    chans = W.noisy_ghz_channels(n_dm, p_dep)[2:4]
    picks = [_LoweredOp(tuple(c.targets) + tuple(t + n_dm for t in c.targets), oracle.dm_superoperator(c.kraus))
             for c in chans]
    return picks, f"dm_ghz{n_dm}", "CNOT / two-qubit depolarising superoperator of noisy GHZ"


def cpu_baseline(n_s: int, seed: int, p: int, workload: str = "qaoa", p_dep: float = 1e-2):
    """Oracle timed on the host (1 thread) on two gates at N = n_s."""
    import oracle
    if workload == "dm_ghz":
        picks, _, what = _dm_oracle_picks(n_s // 2, p_dep)
        n_s = 2 * (n_s // 2)
    elif workload == "wide":
        n_s = min(n_s, 24)
        picks = W.wide_circuit(n_s, n_ops=2, widths=(5, 6), seed=seed)
        what = "2 operators (k=5, k=6) of the wide workload"
    elif workload == "fusion":
        picks = _fusion_picks(n_s, seed)
        what = "2 gates (U(2), U(4)) of the fusion workload"
    else:
        ops, _ = W.qaoa_circuit(n=n_s, p=p, seed=seed)
        picks = [ops[0], ops[n_s]]
        what = "2 gates (H, ZZ) of the QAOA circuit"
    psi = oracle.zero_state(n_s)
    t0 = time.perf_counter()
    for g in picks:
        oracle.apply(psi, g.targets, g.matrix)
    dt = time.perf_counter() - t0
    rate = len(picks) * (1 << n_s) / dt
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{what} at N={n_s}, {dt:.1f} s single-threaded FP64", **host_cpu()}


def step_dtype(agg):
    """The arithmetic the timed steps ran, from the kinds of block they
    applied (not from the options asked for)."""
    ran = []
    if agg["layer_blocks"]:
        ran.append("f32 layer passes")
    if agg["diag_blocks"]:
        ran.append("f32 diagonal passes")
    if agg["prod_blocks"]:
        ran.append("f32 product passes")
    n_fp32 = agg["blocks"] - agg["tc_blocks"] - agg["diag_blocks"] - agg["prod_blocks"] - agg["layer_blocks"]
    if n_fp32:
        ran.append("f32 dense fused products on CUDA cores")
    if agg["tc_blocks"]:
        ran.append("k=5/6 products as 3xTF32 on tensor cores with f32 accumulation")
    if agg["permutes"]:
        ran.append("bit permutations")
    return "c64 state; " + ", ".join(ran) + "; f64 reductions"


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def tc_record(q, torch, buf, stream, n, seed, hbm_peak, n_ops=40):
    """The wide workload's operators at N = n: alternating Haar k = 5 / 6
    operators on random target sets, one pass each, on the split-TF32 tensor
    cores and on the FP32 CUDA cores.  Per precision: ms per operator (CUDA
    events around each launch), operator-level amplitude updates per second
    over the whole run, and the fused kernel's HBM roofline (16 B per
    amplitude per launch)."""
    ops = W.wide_circuit(n, n_ops=n_ops, widths=(5, 6), seed=seed)
    s = q.qsa_state_create_ex(n, buf.data_ptr(), 8 << n, stream, 1)
    out = {"workload": f"wide{n}: {n_ops} Haar k=5/6 operators on random targets, N={n} complex64"}
    try:
        for name, prec in (("tf32x3", q.QSA_PREC_TF32X3), ("fp32", q.QSA_PREC_FP32)):
            plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_PER_GATE, kmax=6, kmax_diag=6,
                                                         precision=prec, timing=1))
            try:
                q.qsa_plan_execute(s, plan)   # warm-up
                e0, e1 = _events(torch)
                torch.cuda.synchronize()
                e0.record()
                st = q.qsa_plan_execute(s, plan)
                e1.record()
                torch.cuda.synchronize()
            finally:
                q.qsa_plan_destroy(plan)
            t = e0.elapsed_time(e1) * 1e-3
            kt = st["tc_seconds"] if prec else st["apply_seconds"]
            per_op = kt / n_ops
            gbs = 16.0 * (1 << n) / per_op / 1e9
            out[name] = {"value": n_ops * float(1 << n) / t, "unit": UNIT, "ms_per_op": per_op * 1e3,
                         "tc_blocks": st["tc_blocks"], "kernel": "k_apply_tc" if prec else "k_apply_fp32",
                         "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                      "frac": gbs / hbm_peak}}
        out["tc_speedup_vs_fp32"] = out["fp32"]["ms_per_op"] / out["tf32x3"]["ms_per_op"]
        # per width: FP32 CUDA-core k = 1..6 and split-TF32 k = 5, 6, 8 operators each on random targets
        per_k = {}
        for name, prec, ks in (("fp32", q.QSA_PREC_FP32, range(1, 7)), ("tf32x3", q.QSA_PREC_TF32X3, (5, 6))):
            for k in ks:
                kops = W.wide_circuit(n, n_ops=8, widths=(k,), seed=seed + 100 + k)
                plan = q.qsa_plan_create(kops, n, q.make_opts(planner=q.QSA_PLAN_PER_GATE, kmax=6, kmax_diag=6,
                                                              precision=prec, timing=1))
                try:
                    q.qsa_plan_execute(s, plan)
                    st = q.qsa_plan_execute(s, plan)
                finally:
                    q.qsa_plan_destroy(plan)
                kt = (st["tc_seconds"] if st["tc_blocks"] else st["apply_seconds"]) / len(kops)
                per_k[f"{name}_k{k}"] = {"ms_per_op": kt * 1e3, "frac": 16.0 * (1 << n) / kt / 1e9 / hbm_peak}
        out["per_width"] = per_k
    finally:
        q.qsa_state_destroy(s)
    return out


def batch_record(q, torch, buf, stream, seed, n=20, n_traj=256, shots=10000, p=1e-3, kmax=4):
    """Batched noisy trajectories: n_traj states of N = n, depths uniform in
    10..60 of U(2) + CZ brick layers with depolarising branches (probability p
    per gate), one persistent launch replayed from a CUDA graph, then shots
    sampled counts per trajectory.  Metrics: trajectories/s and gate-level
    amplitude updates per second (input gates x 2^n per trajectory)."""
    trajs, depths = W.trajectory_batch(n_traj=n_traj, n=n, dmin=10, dmax=60, seed=seed, p=p)
    b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_DP, kmax=kmax, kmax_diag=kmax))
    nbytes = n_traj * (8 << n)
    if buf.numel() * 8 < nbytes:
        buf = torch.empty(nbytes // 8, dtype=torch.complex64, device=buf.device)
    try:
        info = q.qsa_batch_info(b)
        q.qsa_batch_run(b, buf.data_ptr(), nbytes, shots, seed, 0, 1, stream)   # capture + warm-up
        e0, e1 = _events(torch)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0.record()
            st = q.qsa_batch_run(b, buf.data_ptr(), nbytes, shots, seed, 0, 1, stream)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        t = statistics.median(times)
    finally:
        q.qsa_batch_destroy(b)
    gates = sum(len(x) for x in trajs)
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    return {"workload": f"{n_traj} trajectories N={n}, depths 10..60, depolarising p={p:g}, {shots} shots each",
            "kmax": kmax,
            "trajectories_per_s": n_traj / t, "value": gates * float(1 << n) / t, "unit": UNIT,
            "ms_per_batch": t * 1e3, "launch_seconds": st["seconds"], "gates": gates, "fused_blocks": info["blocks"],
            "states_bytes": nbytes, "l2_bytes": l2,
            "bound": "hbm" if nbytes > l2 else "l2",
            "hbm_gbs_if_streamed": info["blocks"] * 16.0 * (1 << n) / t / 1e9}


def planner_record(q, torch, buf, stream, seed, n=28, layers=40, n_samples=1000, precision="tf32x3"):
    """The learned planner against the method without it on the fusion
    workload at N = n: QFT of a seeded basis state, `layers` layers of Haar
    U(2) on every qubit and Haar U(4) on a random matching, then the inverse
    of everything (the state returns to |0...0>).  Plans with kmax 6 and
    diagonal blocks up to 12 qubits: the width-limit heuristic (greedy),
    Eq. dp-recurrence with Gamma = 4^k, and the same DP scored by the cost
    model trained here on this state's own kernel timings.  precision
    "tf32x3" runs k = 5, 6 on the tensor cores (every width then costs about
    one memory pass, the heuristic's own assumption); "fp32" keeps them on the
    CUDA cores, where a 6-qubit block costs several passes.  Each plan's run
    is timed with CUDA events (median of 3)."""
    prec = q.QSA_PREC_TF32X3 if precision == "tf32x3" else q.QSA_PREC_FP32
    ops, _ = W.fusion_circuit(n=n, layers=layers, seed=seed, with_inverse=True)
    if buf.numel() < (1 << n):
        buf = torch.empty(1 << n, dtype=torch.complex64, device=buf.device)
    s = q.qsa_state_create_ex(n, buf.data_ptr(), 8 << n, stream, 1)
    out = {"workload": f"fusion{n}: QFT + {layers} Haar U(2)/U(4) layers + inverse, {len(ops)} gates, "
                       f"N={n} complex64", "kmax": 6, "kmax_diag": 12, "precision": precision}
    try:
        out["cost_model"] = train_cost_model(q, s, prec, seed, n_samples)
        for name, planner in (("greedy", q.QSA_PLAN_GREEDY), ("dp_4k", q.QSA_PLAN_DP),
                              ("dp_mlp", q.QSA_PLAN_DP_MLP)):
            opts = q.make_opts(planner=planner, kmax=6, kmax_diag=12, precision=prec)
            t0 = time.perf_counter()
            plan = q.qsa_plan_create(ops, n, opts)
            plan_s = time.perf_counter() - t0
            try:
                q.qsa_state_reset(s)
                q.qsa_plan_execute(s, plan)   # warm-up
                times = []
                for _ in range(3):
                    q.qsa_state_reset(s)
                    e0, e1 = _events(torch)
                    torch.cuda.synchronize()
                    e0.record()
                    st = q.qsa_plan_execute(s, plan)
                    e1.record()
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1) * 1e-3)
                q.qsa_state_sync(s)
                p0 = float(abs(complex(buf[0].item())) ** 2)   # logical |0...0> sits at index 0 in any layout
            finally:
                blocks = q.qsa_plan_info(plan)["blocks"]
                q.qsa_plan_destroy(plan)
            out[name] = {"seconds": statistics.median(times), "blocks": blocks, "passes": st["passes"],
                         "tc_blocks": st["tc_blocks"], "diag_blocks": st["diag_blocks"], "plan_seconds": plan_s,
                         "return_probability": p0, "value": len(ops) * float(1 << n) / statistics.median(times),
                         "unit": UNIT}
        out["gain_vs_greedy"] = out["greedy"]["seconds"] / out["dp_mlp"]["seconds"]
        out["gain_vs_dp_4k"] = out["dp_4k"]["seconds"] / out["dp_mlp"]["seconds"]
    finally:
        q.qsa_costmodel_set(None)
        q.qsa_state_destroy(s)
    return out


def interleaved_layout(n: int, ways: int = 3):
    """Physical position of logical qubit q: qubits q = g (mod ways) fill the
    g-th block of positions in order.  A run of consecutive qubits (a layer of
    one-qubit gates taken in qubit order) then spreads over low, middle and
    high positions, so no tile of a layer pass holds many of the highest
    positions (each of those spreads a tile over more 2 MiB pages)."""
    sizes = [len(range(g, n, ways)) for g in range(ways)]
    off = [sum(sizes[:g]) for g in range(ways)]
    return [off[q % ways] + q // ways for q in range(n)]


def train_cost_model(q, s, precision, seed, n_samples):
    """Collect timings of the library's own kernels on the bench state, train
    the cost model on the GPU and install it; returns its held-out error."""
    X, y = q.qsa_costmodel_collect(s, n_samples, reps=3, precision=precision, seed=seed + 101)
    perm = np.random.default_rng(seed).permutation(len(y))
    n_tr = int(0.85 * len(y))
    tr, te = perm[:n_tr], perm[n_tr:]
    params, losses = q.qsa_costmodel_train(X[tr], y[tr], epochs=400, batch=32, lr=2e-3, seed=seed + 7,
                                           weight_decay=1e-2)
    q.qsa_costmodel_set(params)
    pred = q.qsa_costmodel_predict(X[te])
    rel = np.abs(pred - np.exp(y[te])) / np.exp(y[te])
    return {"samples": int(len(y)), "heldout_median_rel_err": float(np.median(rel)),
            "final_loss": float(losses[-1])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qaoa", choices=["qaoa", "dm_ghz", "wide", "fusion"],
                    help="qaoa: the N=30 QAOA circuit; dm_ghz: noisy GHZ density matrix; wide: --wide-ops Haar "
                         "k=5/6 operators on random targets, one pass each (--precision picks the tensor-core or "
                         "CUDA-core path); fusion: QFT + Haar U(2)/U(4) layers + inverse, planned like the QAOA "
                         "step (dense blocks up to k = 6, split-TF32 for k = 5, 6)")
    ap.add_argument("--wide-ops", type=int, default=40, help="operators per step of --workload wide")
    ap.add_argument("--fusion-layers", type=int, default=40,
                    help="Haar U(2)/U(4) layers of --workload fusion (QFT + layers + inverse; use --n 28 for the "
                         "N=28 fusion configuration)")
    ap.add_argument("--dm-n", type=int, default=15, help="density-matrix qubits of --workload dm_ghz (2..17)")
    ap.add_argument("--dm-p", type=float, default=1e-2, help="depolarising rate of --workload dm_ghz")
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--shots", type=int, default=1000)
    ap.add_argument("--planner", default="dp_mlp", choices=["per_gate", "greedy", "dp", "dp_mlp"])
    ap.add_argument("--kmax", type=int, default=6)
    ap.add_argument("--kmax-diag", type=int, default=12, help="diagonal-block cap (1..12)")
    ap.add_argument("--kmax-prod", type=int, default=0, help="product-unit cap (0: off, 2..11)")
    ap.add_argument("--layer", type=int, default=1, choices=[0, 1],
                    help="1: layer units (diagonal gates + one-qubit factors in one tile pass)")
    ap.add_argument("--zero-init", type=int, default=1, choices=[0, 1],
                    help="1: the circuit's product-state prefix on |0...0> in one write-only pass")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3"])
    ap.add_argument("--lowering", default="auto", choices=["auto", "strided", "permute"])
    ap.add_argument("--victim", default="first_free", choices=["first_free", "farthest"],
                    help="eviction rule of --lowering permute promotions")
    ap.add_argument("--layout", default="interleave", choices=["identity", "interleave"],
                    help="initial layout, set on |0...0> as a metadata-only relabel before each step")
    ap.add_argument("--cm-samples", type=int, default=1000, help="timings the cost model of the bench plan trains on")
    ap.add_argument("--ref-qubits", type=int, default=28)
    ap.add_argument("--cpu-qubits", type=int, default=28)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the per-gate comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-n", type=int, default=20, help="qubits per trajectory of the batch sub-record")
    ap.add_argument("--batch-traj", type=int, default=256, help="trajectories of the batch sub-record")
    ap.add_argument("--batch-kmax", type=int, default=4, choices=[1, 2, 3, 4], help="fused-block cap of the batch sub-record")
    ap.add_argument("--records", default="tc,planner,batch",
                    help="comma list of sub-records measured after the timed region on rank 0 "
                         "(tc: split-TF32 vs FP32 k=5/6 operators at N=30; planner: greedy / 4^k DP / learned DP "
                         "on the N=28 fusion circuit; batch: 256 noisy trajectories at N=20); "
                         "'' for none")
    args = ap.parse_args()

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2608_16940_gb300 as q

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    dm = args.workload == "dm_ghz"
    wide = args.workload == "wide"
    fusion = args.workload == "fusion"
    if wide:
        # each operator is one fused block already (k = 5, 6): no fusion, no layer units, no cost model
        args.planner, args.layer, args.zero_init, args.layout = "per_gate", 0, 0, "identity"
    if dm:
        n_dm = args.dm_n
        n = 2 * n_dm
        chans = W.noisy_ghz_channels(n_dm, args.dm_p)
        ops = [q.qsa_dm_superoperator(n_dm, c.targets, c.kraus) for c in chans]
        edges = [(0, n_dm - 1)]
    elif wide:
        n = args.n
        ops = W.wide_circuit(n, n_ops=args.wide_ops, widths=(5, 6), seed=args.seed + rank)
        edges = [(0, 1)]
    elif fusion:
        n = args.n
        ops, _ = W.fusion_circuit(n=n, layers=args.fusion_layers, seed=args.seed + rank, with_inverse=True)
        edges = [(0, 1)]
    else:
        n = args.n
        ops, edges = W.qaoa_circuit(n=n, p=args.p, seed=args.seed + rank)
    planner = {"per_gate": 0, "greedy": 1, "dp": 2, "dp_mlp": 3}[args.planner]
    prec = {"fp32": 0, "tf32x3": 1}[args.precision]
    low = {"auto": 0, "strided": 1, "permute": 2}[args.lowering]
    kdiag = args.kmax_diag
    victim = {"first_free": 0, "farthest": 1}[args.victim]
    opts = q.make_opts(planner=planner, kmax=args.kmax, kmax_diag=kdiag, precision=prec, lowering=low, timing=1,
                       victim=victim, kmax_prod=args.kmax_prod, layer=args.layer, zero_init=args.zero_init)
    # the same plan without per-launch timing, as a user builds it (end-to-end measurement)
    opts_user = q.make_opts(planner=planner, kmax=args.kmax, kmax_diag=kdiag, precision=prec, lowering=low,
                            victim=victim, kmax_prod=args.kmax_prod, layer=args.layer, zero_init=args.zero_init)

    buf = torch.empty(1 << n, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    s = q.qsa_state_create_ex(n, buf.data_ptr(), buf.numel() * 8, stream, 1)
    cm = None
    if planner == 3:
        cm = train_cost_model(q, s, prec, args.seed, args.cm_samples)
        q.qsa_state_reset(s)
    layout = interleaved_layout(n) if args.layout == "interleave" else None
    plan = q.qsa_plan_create(ops, n, opts, layout=layout)

    def reset():
        q.qsa_state_reset(s)
        if layout is not None:
            q.qsa_set_layout(s, layout, 0)   # |0...0>: relabel only, no data moves
    pinfo = q.qsa_plan_info(plan)
    edge_mask = (1 << edges[0][0]) | (1 << edges[0][1])

    agg = {"apply_seconds": 0.0, "tc_seconds": 0.0, "permute_seconds": 0.0, "diag_seconds": 0.0,
           "prod_seconds": 0.0, "layer_seconds": 0.0, "blocks": 0, "passes": 0, "permutes": 0, "tc_blocks": 0,
           "diag_blocks": 0, "prod_blocks": 0, "layer_blocks": 0}

    def step(record):
        st = q.qsa_plan_execute_from_zero(s, plan)   # |0...0> in the plan's layout, then the plan
        if dm:
            norm = q.qsa_dm_probabilities(s, n_dm, want_probs=False)[1]
            zz = q.qsa_dm_expectation_z(s, n_dm, edge_mask)
            nshot = 0
        else:
            # norm, <Z_a Z_b> and the shots from one read of the state
            (norm, zz), vals, cnts = q.qsa_measure(s, [0, edge_mask], args.shots, seed=args.seed + 17)
            nshot = int(cnts.sum())
        if record:
            for k in agg:
                agg[k] += st[k]
        return norm, zz, nshot

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    l0 = q.qsa_state_counters(s)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("qsa_timed")
    t_wall0 = time.time()
    ev0.record()
    for _ in range(args.steps):
        norm, zz, nshot = step(True)
    ev1.record()
    torch.cuda.synchronize()
    t_wall1 = time.time()
    torch.cuda.nvtx.range_pop()
    launches = q.qsa_state_counters(s) - l0
    clocks = clk.stop(t_wall0, t_wall1)
    elapsed = job_seconds(ev0.elapsed_time(ev1) * 1e-3, ws, dev)
    per_step = elapsed / args.steps
    amp_updates = len(ops) * float(1 << n)
    value = job_value(amp_updates, ws, per_step)

    # roofline of the dominant fused-operator kernel: 16 B per amplitude per launch
    hbm_peak, peak_kind = _peaks()
    bytes_per_launch = 16.0 * (1 << n)
    n_fp32 = agg["blocks"] - agg["tc_blocks"] - agg["diag_blocks"] - agg["prod_blocks"] - agg["layer_blocks"]
    kinds = []
    if n_fp32:
        kinds.append(("k_apply_fp32 (FP32 fused dense update)", agg["apply_seconds"], n_fp32))
    if agg["tc_blocks"]:
        kinds.append(("k_apply_tc (split-TF32 tcgen05 fused update)", agg["tc_seconds"], agg["tc_blocks"]))
    if agg["diag_blocks"]:
        kinds.append(("k_apply_diag (diagonal streaming update)", agg["diag_seconds"], agg["diag_blocks"]))
    if agg["prod_blocks"]:
        kinds.append(("k_apply_prod (product of one-qubit factors)", agg["prod_seconds"], agg["prod_blocks"]))
    if agg["layer_blocks"]:
        # one pass per layer block unless its factors need more than one tile
        n_layer_pass = agg["passes"] - agg["permutes"] - (agg["blocks"] - agg["layer_blocks"])
        kinds.append(("k_apply_layer (diagonal gates + one-qubit factors, one tile pass)", agg["layer_seconds"],
                      n_layer_pass))
    if agg["permutes"]:
        kinds.append(("k_permute (qubit permutation)", agg["permute_seconds"], agg["permutes"]))
    name, tot, cnt = max(kinds, key=lambda kv: kv[1])
    avg = tot / cnt
    kernel_bytes = bytes_per_launch * cnt
    if name.startswith("k_apply_layer"):
        # zero-state preparation passes only write (8 B per amplitude)
        kernel_bytes -= bytes_per_launch / 2 * q.qsa_plan_block_kinds(plan)[0].count(4) * args.steps
    achieved = kernel_bytes / tot / 1e9
    dram = DRAM_BYTES_PER_AMP.get(name.split(" ")[0])
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": dram * (1 << n) if dram else None, "kernel": name, "peak_source": peak_kind, "bytes_per_launch": kernel_bytes / cnt,
            "avg_launch_ms": avg * 1e3, "launches_per_step": cnt / args.steps,
            "share_of_step": tot / args.steps / per_step}

    # end to end through the public API from host data: plan + upload + apply + the step's norm, <ZZ>
    # and counts copied back
    e2e = None
    if not args.no_e2e:
        e2e_times = []
        h2d = d2h = 0.0
        for _ in range(max(1, min(3, args.steps))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # the plan from the host op list (fusion, FP64 block products, FP32 constants), its upload, and
            # the run from |0...0> (cleared first unless the plan's first pass writes every amplitude)
            p_e2e = q.qsa_plan_create(ops, n, opts_user, layout=layout)
            try:
                st = q.qsa_plan_execute_from_zero(s, p_e2e)
            finally:
                q.qsa_plan_destroy(p_e2e)
            if dm:
                q.qsa_dm_probabilities(s, n_dm, want_probs=False)
                q.qsa_dm_expectation_z(s, n_dm, edge_mask)
                d2h = 16.0
            else:
                _, vals, cnts = q.qsa_measure(s, [0, edge_mask], args.shots, seed=args.seed + 17)
                d2h = 16.0 * len(vals) + 16 + 16
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
            h2d = st["h2d_bytes"]
        e2e = {"value": ws * amp_updates / statistics.median(e2e_times), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    extra = {}
    if not args.no_compare and rank == 0:
        # plain per-gate comparator on the same state and circuit (one step)
        pg = q.qsa_plan_create(ops, n, q.make_opts(planner=0, kmax=2, kmax_diag=2, timing=1))
        q.qsa_state_reset(s)
        q.qsa_plan_execute(s, pg)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        q.qsa_state_reset(s)
        e0.record()
        pst = q.qsa_plan_execute(s, pg)
        e1.record()
        torch.cuda.synchronize()
        pg_t = e0.elapsed_time(e1) * 1e-3
        q.qsa_plan_destroy(pg)
        extra["per_gate"] = {"value": amp_updates / pg_t, "unit": UNIT, "seconds": pg_t, "passes": pst["passes"],
                             "hbm_gbs": pst["passes"] * bytes_per_launch / pg_t / 1e9,
                             "fused_speedup": (amp_updates / per_step) / (amp_updates / pg_t)}

    recs = [r for r in args.records.split(",") if r] if (rank == 0 and not dm and not wide and not fusion) else []
    if "tc" in recs:
        extra["tc"] = tc_record(q, torch, buf, stream, n, args.seed, hbm_peak)
    if "planner" in recs:
        extra["planner"] = planner_record(q, torch, buf, stream, args.seed)
        extra["planner_fp32"] = planner_record(q, torch, buf, stream, args.seed, precision="fp32")
    if "batch" in recs:
        extra["batch"] = batch_record(q, torch, buf, stream, args.seed, n=args.batch_n, n_traj=args.batch_traj,
                                      kmax=args.batch_kmax)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_qubits, args.seed, args.p, args.workload, args.dm_p)

    q.qsa_costmodel_set(None)
    q.qsa_plan_destroy(plan)
    q.qsa_state_destroy(s)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": step_dtype(agg),
                "data": "synthetic",
                "config": {"workload": (f"wide{n}: {len(ops)} Haar k=5/6 operators on random targets, N={n} "
                                        f"complex64 ({8 * (1 << n) / 2**30:g} GiB), from |0...0> (reset included), "
                                        f"norm + <Z0 Z1> + {args.shots} shots per step") if wide else
                                       (f"dm_ghz{n_dm}: noisy GHZ density matrix, {len(ops)} channels "
                                        f"(depolarising p={args.dm_p:g} after each gate) lowered to superoperators, "
                                        f"vec(rho) on 2n={n} qubits complex64 ({8 * (1 << n) / 2**30:g} GiB), "
                                        f"trace + Tr(rho Z0 Z{n_dm - 1}) per step") if dm else
                                       (f"fusion{n}: QFT of a seeded basis state + {args.fusion_layers} Haar U(2)/U(4) "
                                        f"layers + the inverse of everything, {len(ops)} gates, N={n} complex64 "
                                        f"({8 * (1 << n) / 2**30:g} GiB), returns to |0...0>; norm + <Z0 Z1> + "
                                        f"{args.shots} shots per step") if fusion else
                                       (f"qaoa{n}_p{args.p}: random 3-regular graph, {len(ops)} gates, N={n} "
                                        f"complex64 ({8 * (1 << n) / 2**30:g} GiB), {args.shots} shots + norm + "
                                        f"<ZZ> per step"),
                           "planner": args.planner, "kmax": args.kmax, "kmax_diag": kdiag,
                           "kmax_prod": args.kmax_prod, "layer": args.layer, "zero_init": args.zero_init,
                           "precision": args.precision,
                           "lowering": args.lowering, "victim": args.victim, "fused_blocks": pinfo["blocks"],
                           "layout": args.layout,
                           "l2": (f"state {8 * (1 << n) / 2**30:g} GiB > L2 "
                                  f"{torch.cuda.get_device_properties(dev).L2_cache_size / 2**20:.0f} MiB; no flush needed"
                                  if (8 << n) > torch.cuda.get_device_properties(dev).L2_cache_size else
                                  "state smaller than L2: timings include L2 reuse"),
                           "parallelism": f"replicas x{ws}"},
                "gpu_launches": launches, "clocks": clocks, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "passes_per_step": agg["passes"] / args.steps,
                "hbm_gbs_step": agg["passes"] / args.steps * bytes_per_launch / per_step / 1e9,
                "cost_model": cm, "check": {"norm": norm, "zz_edge0": zz, "shots": nshot}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
