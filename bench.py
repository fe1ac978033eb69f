#!/usr/bin/env python
"""Throughput of the batched PAAM WCRT analysis (Sec. IV-F, Theorem 1) on GB300.

One step = one exact analysis of every chain of the 1,000,000-system workload
(8-16 chains of 3-8 callbacks, 4 executors on 2 cores, utilisation swept
0.3..0.9, accelerator-segment probability 0.5), inputs resident in HBM.
Prints one JSON line.  ``--impl reference`` times the plain CPU oracle on the
host cores instead (the reference arm: there is no reference implementation
to run, so the oracle stands in for it).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "analysed chains/sec (bit-exact WCRT) and priority-search systems/sec, surrogate vs plain"
WORKLOAD = "cfg2"
WORKLOAD_DESC = ("1,000,000 synthetic ROS 2 systems: 8-16 chains of 3-8 callbacks, 4 executors on 2 cores "
                 "plus the PAAM server, utilisation swept 0.3-0.9, accelerator-segment probability 0.5 "
                 "(0.1-2 ms), periods log-uniform 10-100 ms, D = T, one accelerator, n_buckets = 1, "
                 "eps = kappa = 0; int64 ns")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-sys", type=int, default=None, help="override the workload size (testing)")
    ap.add_argument("--no-search", action="store_true", help="skip the priority-search measurements")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurements")
    ap.add_argument("--search-sys", type=int, default=10_000)
    ap.add_argument("--train-sys", type=int, default=10_000_000, help="systems the surrogate trains on")
    ap.add_argument("--top-k", type=int, default=16)
    ap.add_argument("--gemm", type=int, nargs=3, default=None, metavar=("M", "N", "K"),
                    help="time only the tensor-core GEMM C[M,N] = A[M,K] B[N,K]^T")
    ap.add_argument("--infer", type=int, default=None, metavar="N_SYS",
                    help="time only the network's ranking of 256 candidate orders of N_SYS search systems")
    ap.add_argument("--kappa", type=int, default=None, metavar="ITERS",
                    help="only measure the device preemption cost, ITERS iterations per kernel kind")
    ap.add_argument("--kappa-iters", type=int, default=300, help="preemption-cost iterations in the full run")
    ap.add_argument("--launch-config", type=int, default=None, help="fixed launch configuration (no autotune)")
    ap.add_argument("--workload", default="cfg2", choices=["cfg1", "cfg2", "cfg3"],
                    help="the analysis workload of the timed step (default: the 1M-system one)")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other analysis workloads (cfg1, cfg3)")
    ap.add_argument("--workload-steps", type=int, default=20, help="timed steps of each other workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons, loaded = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 11:
                continue
            try:
                clk, cmax, util = float(r[2]), float(r[3]), float(r[5])
            except ValueError:
                continue
            sm.append(clk)
            smax.append(cmax)
            if util >= 50:
                loaded.append(clk)
                for nm, v in zip(names, r[7:11]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        use = loaded or sm
        return {"sm_mhz": float(np.median(use)) if use else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(loaded)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo; architecture otherwise)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


# main kernel of each launch configuration (the table in csrc/analyze_fast.cu)
# the passes over the first pass's deferral list, launched only for a batch with systems
# above 16 chains (or deferred for their deadlines)
_REG_BIG = "; analyze_reg_kernel<32, 2> for the deferred systems"
_LAZY_BIG = ("; analyze_lazy_kernel<32, 6> for the deferred systems of up to 32 chains and "
             "analyze_lazy64_kernel<3> for those above")
CONFIG_KERNEL = {0: "analyze_reg_kernel<8, 2>", 1: "analyze_fast_kernel<8, 16>", 2: "analyze_fast_kernel<16, 32>",
                 3: "analyze_reg1_kernel<16>", 4: "analyze_reg_kernel<4, 4>", 5: "analyze_reg_kernel<16, 2>",
                 6: "analyze_reg1_kernel<32>", 7: "analyze_reg_kernel<8, 2>", 8: "analyze_fast_kernel<4, 16>",
                 9: "analyze_fast_kernel<8, 32>", 10: "analyze_reg_kernel<16, 2>", 11: "analyze_reg_kernel<4, 4>",
                 12: "analyze_reg1_kernel<16> (work queue)", 13: "analyze_reg_kernel<8, 2> (work queue)",
                 14: "analyze_fast_kernel<8, 16> (work queue)", 15: "analyze_reg_kernel<16, 2> (work queue)",
                 16: "analyze_reg1_kernel<32> (work queue)", 17: "analyze_reg1_kernel<16> (work queue, size-binned)",
                 18: "analyze_reg1_kernel<32> (work queue, size-binned)",
                 19: "analyze_reg_kernel<8, 2> (work queue, size-binned)",
                 20: "analyze_lazy_kernel<16, 4>" + _REG_BIG, 21: "analyze_lazy_kernel<16, 4> (work queue)" + _REG_BIG,
                 22: "analyze_lazy_kernel<16, 4> (work queue, size-binned)" + _REG_BIG,
                 23: "analyze_lazy_kernel<16, 5> (work queue, size-binned)" + _REG_BIG,
                 24: "analyze_lazy_kernel<16, 6> (work queue, size-binned)" + _REG_BIG,
                 25: "analyze_lazy_kernel<16, 5> (work queue)" + _REG_BIG,
                 26: "analyze_lazy_kernel<16, 6> (work queue, size-binned)" + _LAZY_BIG,
                 27: "analyze_lazy_kernel<16, 4> (work queue, size-binned)" + _LAZY_BIG,
                 28: "analyze_lazy_kernel<16, 5> (work queue, size-binned)" + _LAZY_BIG}


# DRAM read + write per system of the analysis kernels, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) of 500,000 systems of a
# workload, per launch configuration, and the executed warp-instructions per
# system of the same captures (smsp__inst_executed.sum / 500,000 systems): the
# instruction-issue side, against the issue peak of 152 SMs x 4 schedulers x 1
# per clock.  Valid only while the kernels and the order they visit are
# unchanged since the capture; a configuration without an entry reports null.
# 26: analyze_lazy_kernel<16, 6> (1,022.1 MB), 28: analyze_lazy_kernel<16, 5> (959.0 MB);
# neither defers a system of this workload, so configurations 24 and 23 run the
# same kernels in the same order on it and take the same entries.
_T26, _T28 = (949_534_464 + 72_603_904) / 500_000, (901_364_736 + 57_655_808) / 500_000
TRAFFIC_PER_SYSTEM = {26: _T26, 24: _T26, 28: _T28, 23: _T28}
# the same for the other workloads, keyed by (workload, launch configuration): the
# uneven workload's step is the first pass, the 32-lane pass over the deferral list
# and the 64-chain lazy kernel for the systems above 32 chains
TRAFFIC_OTHER = {("cfg3", 26): (867_346_688 + 40_391_936 + 346_479_616 + 16_131_584 + 109_261_824 + 1_899_520) / 500_000,
                 ("cfg3", 28): (849_617_152 + 30_518_528 + 346_491_904 + 16_272_896 + 109_204_480 + 1_914_624) / 500_000}


def traffic_per_system(workload: str, cfg_index: int):
    if workload == "cfg2":
        return TRAFFIC_PER_SYSTEM.get(cfg_index)
    return TRAFFIC_OTHER.get((workload, cfg_index))


WARP_INST_PER_SYSTEM = {26: 551_079_382 / 500_000, 24: 551_079_382 / 500_000, 28: 531_338_213 / 500_000,
                        23: 531_338_213 / 500_000}
ISSUE_PEAK = 152 * 4 * 2.07e9  # warp-instructions / s at the 2070 MHz maximum SM clock


def algorithmic_bytes(sy) -> int:
    """Bytes one analysis must move: every input table read once (the
    accelerator index is not kept: one accelerator) plus R, status, verdict."""
    inp = (sy.sys_chain_off.nbytes + sy.chain_cb_off.nbytes + sy.cb_seg_off.nbytes + sy.T.nbytes + sy.D.nbytes
           + sy.prio.nbytes + sy.exec.nbytes + sy.spin.nbytes + sy.E.nbytes + sy.A.nbytes + sy.sys_exec_off.nbytes
           + sy.exec_core.nbytes + (sy.exec_prio.nbytes if sy.exec_prio is not None else 0))
    out = sy.n_chain * 9 + sy.n_sys
    return int(inp + out)


# The other analysis workloads, each timed as the headline one is (one step =
# one graph replay of the autotuned analysis of the whole batch, inputs
# resident), with its own roofline, end-to-end call and oracle baseline.
EXTRA_WORKLOADS = {
    "cfg1": dict(desc="1,000 systems: 4 chains of 2-4 callbacks, 2 executors on 1 core, one accelerator, "
                      "utilisation 0.5, segment probability 0.3; n_buckets = 1, eps = kappa = 0; int64 ns",
                 cpu_sample=None, flush_l2=True, params=dict(n_buckets=1, eps=0, kappa=0)),
    "cfg3": dict(desc="4,000,000 systems of uneven size: 2 + Geom(1/9) chains (<= 64), 1-12 callbacks, "
                      "2-8 executors, utilisation U[0.2, 0.95], segment probability 0.5; n_buckets = 1, "
                      "eps = kappa = 0; int64 ns; one CUDA-graph replay of the autotuned persistent launch "
                      "(size-binned work queue, deferral of larger systems) per step",
                 cpu_sample=200_000, flush_l2=False, params=dict(n_buckets=1, eps=0, kappa=0)),
}
L2_BYTES = 129 * 1024 * 1024


def workload_bench(pkg, ctx, cfg, steps, warmup, e2e_steps, with_cpu):
    """Throughput, roofline, end-to-end call and oracle baseline of one more
    analysis workload (see EXTRA_WORKLOADS)."""
    import torch

    import paam_gen

    w = EXTRA_WORKLOADS[cfg]
    sy = paam_gen.generate(cfg)
    stream = torch.cuda.Stream()
    batch = pkg.paam_rta_load_systems(ctx, sy, stream=stream)
    opts = pkg.analysis_opts(**w["params"])
    cfg_index, _ = pkg.paam_rta_autotune(ctx, batch, opts, stream=stream)
    R = torch.empty(batch.n_chain, dtype=torch.int64, device="cuda")
    st = torch.empty(batch.n_chain, dtype=torch.uint8, device="cuda")
    v = torch.empty(batch.n_sys, dtype=torch.uint8, device="cuda")
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda") if w["flush_l2"] else None
    step = lambda: pkg.paam_rta_analyze_batch(ctx, batch, opts, R, st, v, stream=stream)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        if flush is not None:  # inputs smaller than L2: evict them between steps (untimed)
            with torch.cuda.stream(stream):
                flush.random_(0, 255)
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.launch_count() - launches0
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))
    alg = algorithmic_bytes(sy)
    pk = peaks()
    traffic = traffic_per_system(cfg, cfg_index)
    out = {"workload": w["desc"], "systems": sy.n_sys, "chains": sy.n_chain, "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "chains_per_s": sy.n_chain / (ms / 1e3), "systems_per_s": sy.n_sys / (ms / 1e3),
           "launch_config": cfg_index, "kernel": CONFIG_KERNEL.get(cfg_index, "analysis kernel"),
           "gpu_launches": int(launches),
           "l2": "L2 flushed before every step (inputs %.1f MB)" % (sy.nbytes() / 1e6) if flush is not None
           else "inputs larger than L2 (%.2f GB)" % (sy.nbytes() / 1e9),
           "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "peak_src": pk["src"],
                        "traffic": None if traffic is None else traffic * sy.n_sys,
                        "algorithmic_bytes_per_launch": alg,
                        "scope": "every kernel of the step (the analysis graph), algorithmic bytes of the batch"}}
    # end to end through the C ABI with page-locked host buffers
    pinned = pkg.to_device(sy, pin=True)
    hR = torch.empty(batch.n_chain, dtype=torch.int64).pin_memory()
    hst = torch.empty(batch.n_chain, dtype=torch.uint8).pin_memory()
    hv = torch.empty(batch.n_sys, dtype=torch.uint8).pin_memory()
    h2d = sum(getattr(pinned, f).numel() * getattr(pinned, f).element_size()
              for f in ["sys_chain_off", "chain_cb_off", "cb_seg_off", "T", "D", "prio", "exec", "spin", "E",
                        "A", "acc", "sys_exec_off", "exec_core", "exec_prio"] if getattr(pinned, f) is not None)
    e2e_step = lambda: pkg.paam_rta_analyze_host(ctx, pinned, opts, hR, hst, hv, launch_config=cfg_index)
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    dt = (time.perf_counter() - t0) / e2e_steps
    out["e2e"] = {"value": sy.n_chain / dt, "unit": "chains/s", "ms_per_step": dt * 1e3, "steps": e2e_steps,
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hR.numel() * 9 + hv.numel())}
    same_host = bool(torch.equal(hR, R.cpu()) and torch.equal(hst, st.cpu()) and torch.equal(hv, v.cpu()))
    out["e2e"]["same_results_as_device_path"] = same_host
    if with_cpu:
        import oracle

        cores = os.cpu_count() or 1
        idx = np.arange(sy.n_sys if w["cpu_sample"] is None else min(w["cpu_sample"], sy.n_sys))
        sub = sy.subset(idx)
        t0 = time.perf_counter()
        ref = oracle.analyze(sub, threads=cores, **w["params"])
        dt = time.perf_counter() - t0
        ci = sy.chain_index(idx)
        same = bool(np.array_equal(ref["R"], R.cpu().numpy()[ci]) and
                    np.array_equal(ref["status"], st.cpu().numpy()[ci]) and
                    np.array_equal(ref["verdict"], v.cpu().numpy()[idx]))
        out["cpu_baseline"] = {"value": sub.n_chain / dt, "unit": "chains/s", "cores": cores, "kind": "oracle",
                               "sample": ("the whole workload" if w["cpu_sample"] is None else
                                          f"the first {len(idx)} systems of the workload ({sub.n_chain} chains)"),
                               "systems_per_s": len(idx) / dt, "bit_exact_vs_gpu": same}
    out["status_fractions"] = [float((st == k).float().mean()) for k in range(3)]
    batch.free()
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import paam_gen

    n_sys = args.n_sys or paam_gen.CONFIGS[WORKLOAD]["n_sys"]
    sy = paam_gen.generate(WORKLOAD, n_sys=n_sys)
    cores = os.cpu_count() or 1
    sample = min(20_000, n_sys)
    n_slices = max(1, n_sys // sample)

    slices = {}

    def step(i):
        k = i % n_slices
        if k not in slices:
            slices[k] = sy.subset(np.arange(k * sample, (k + 1) * sample))
        sub = slices[k]
        t = time.perf_counter()
        oracle.analyze(sub, threads=cores)
        return sub.n_chain, time.perf_counter() - t

    for i in range(args.warmup):
        step(i)
    dt = 0.0
    chains = 0
    for i in range(args.steps):
        n, t = step(args.warmup + i)
        chains += n
        dt += t
    val = chains / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "chains/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "step": f"{sample} systems of the workload per step"},
        "cpu_baseline": {"value": val, "unit": "chains/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample}-system slices of the {n_sys}-system workload, one per step",
                         "cpu_model": cpu_model()},
        "e2e": {"value": val, "unit": "chains/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# priority search (256 candidate orders per system) and the surrogate
# ---------------------------------------------------------------------------
SEARCH_K = 256
# guided search: the two heuristic seeds (slots 0 and 1) are always confirmed,
# the network ranks the rest
SEARCH_PINNED = 2


def _timed(fn, reps=1):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps, out


def search_candidates(pkg, ctx, sy, b, cfg):
    """The search workload's SEARCH_K candidate orders per system, on the
    device: slot 0 the Audsley-style seed computed by the library on the GPU,
    slot 1 deadline-monotonic, slots 2.. seeded random permutations.  Returns
    (ranks, seconds the seed took)."""
    import torch

    import paam_gen

    ranks = paam_gen.candidate_ranks(sy, SEARCH_K, paam_gen.CONFIGS[cfg]["seed"] + 7)
    r = torch.from_numpy(ranks).cuda()
    pkg.audsley_order(ctx, b, r.shape[2])  # warm-up
    t, seed = _timed(lambda: pkg.audsley_order(ctx, b, r.shape[2]))
    r[:, 0, :] = seed
    return r, t


def search_bench(pkg, ctx, n_sys):
    """Exhaustive and early-exit exact search on the specified search workload
    (cfg4) and on its sparse-executor variant (cfg4s)."""
    import paam_gen

    out = {}
    for cfg in ("cfg4", "cfg4s"):
        sy = paam_gen.generate(cfg, n_sys=n_sys)
        b = pkg.paam_rta_load_systems(ctx, sy)
        r, t_seed = search_candidates(pkg, ctx, sy, b, cfg)
        # each mode in the launch shape the search autotuner picks for it
        cfg_x, _ = pkg.paam_rta_autotune_search(ctx, b, pkg.analysis_opts(), r)
        pkg.search(ctx, b, r)  # warm-up
        t_x, (first, cand) = _timed(lambda: pkg.search(ctx, b, r), 3)
        cfg_e, _ = pkg.paam_rta_autotune_search(ctx, b, pkg.analysis_opts(), r, stop_at_first=True)
        t_e, (first_e, _) = _timed(lambda: pkg.search(ctx, b, r, stop_at_first=True, want_cand_ok=False), 3)
        cand_np = cand.cpu().numpy()
        assert np.array_equal(first.cpu().numpy(), first_e.cpu().numpy())
        out[cfg] = {
            "systems": sy.n_sys, "candidates_per_system": SEARCH_K,
            "exhaustive_systems_per_s": sy.n_sys / t_x, "exhaustive_ms": t_x * 1e3,
            "early_exit_systems_per_s": sy.n_sys / t_e, "early_exit_ms": t_e * 1e3,
            "candidate_analyses_per_s": sy.n_sys * SEARCH_K / t_x,
            "systems_with_schedulable_order": float((first.cpu().numpy() >= 0).mean()),
            "schedulable_candidates": float(cand_np.mean()),
            "launch_config": {"exhaustive": cfg_x, "early_exit": cfg_e},
            "audsley_seed_ms": t_seed * 1e3,
            "audsley_seed_admitted": float(cand_np[:, 0].mean()),
            "deadline_monotonic_admitted": float(cand_np[:, 1].mean()),
        }
        b.free()
    return out


def _random_orders(sy, seed):
    """The systems' priorities replaced by seeded random permutations (CAPA executor priorities)."""
    rng = np.random.default_rng(seed)
    n = sy.chains_per_system()
    keys = rng.random(sy.n_chain) + np.repeat(np.arange(sy.n_sys), n)  # sort within each system
    order = np.argsort(keys, kind="stable")
    local = np.empty(sy.n_chain, np.int64)
    local[order] = np.arange(sy.n_chain) - np.repeat(sy.sys_chain_off[:-1], n)
    sy.prio = local.astype(np.int32)
    sy.exec_prio = None
    return sy


# training recipe: chunks of 1M systems cycling through these generators (the
# search workload's shape twice per cycle, with random priority orders), each
# chunk trained for TRAIN_EPOCHS passes
TRAIN_SOURCES = ("cfg4s", "cfg2", "cfg4s", "cfg3")
TRAIN_EPOCHS, TRAIN_LR = 3, 2e-3


def surrogate_bench(pkg, ctx, train_sys, n_search, top_k, epochs=TRAIN_EPOCHS, lr=TRAIN_LR, sources=TRAIN_SOURCES):
    """Train the ranking network on exactly analysed systems, then compare the
    guided search (network ranking + exact confirmation of the top-k) with the
    exhaustive exact search on the same candidates."""
    import torch

    import paam_gen

    # the method's own flops: training runs the full 1,024-wide first layer forward,
    # and backward the weight gradients of every layer plus the input gradients of
    # layers 2-4; the ranking reads 16 features for each of a system's chains, so its
    # first layer has K = 16 x (largest chain count), rounded up to 64 (256 for 16-chain systems)
    fwd = lambda kx: 2.0 * (kx * 256 + 256 * 256 + 256 * 256 + 256 * 64)
    flops_train_row = fwd(1024) + fwd(1024) + 2.0 * (256 * 256 + 256 * 256 + 256 * 64)
    sources = tuple(sources)
    chunk = 1_000_000
    model, t_train, t_label, losses, rows = None, 0.0, 0.0, [], 0
    for i, lo in enumerate(range(0, train_sys, chunk)):
        n = min(chunk, train_sys - lo)
        cfg = sources[i % len(sources)]
        sy = paam_gen.generate(cfg, n_sys=n, seed=paam_gen.CONFIGS[cfg]["seed"] + 1000 + i)
        if cfg == "cfg4s":
            sy = _random_orders(sy, i)
        b = pkg.paam_rta_load_systems(ctx, sy)
        dt, (R, st, _) = _timed(lambda: pkg.analyze(ctx, b))
        t_label += dt
        loss = np.zeros(epochs, np.float32)
        opts = pkg.train_opts(epochs=epochs, batch_rows=8192, lr=lr, seed=i, epoch_loss=loss)
        dt, model = _timed(lambda: pkg.paam_surrogate_train(ctx, b, R, st, opts, model))
        t_train += dt
        losses.append(round(float(loss[-1]), 5))
        rows += n
        b.free()
    # held-out error of the predicted R/D on each training source
    mae = {}
    for cfg in dict.fromkeys(sources):
        sy = paam_gen.generate(cfg, n_sys=50_000, seed=paam_gen.CONFIGS[cfg]["seed"] + 999)
        if cfg == "cfg4s":
            sy = _random_orders(sy, 999)
        b = pkg.paam_rta_load_systems(ctx, sy)
        R, st, _ = pkg.analyze(ctx, b)
        pred = torch.empty((sy.n_sys, 64), dtype=torch.float32, device="cuda")
        pkg.paam_surrogate_predict(ctx, model, b, pred)
        torch.cuda.synchronize()
        Rn, stn = R.cpu().numpy(), st.cpu().numpy()
        y = np.where(stn == 0, np.minimum(np.maximum(Rn, 0) / sy.D, 2.0), 2.0)
        n = sy.chains_per_system()
        sysid = np.repeat(np.arange(sy.n_sys), n)
        p = pred.cpu().numpy()[sysid, np.arange(sy.n_chain) - sy.sys_chain_off[sysid]]
        mae[cfg] = round(float(np.abs(p - y).mean()), 5)
        b.free()

    # the search workload: SEARCH_K candidate orders per system
    K = SEARCH_K
    sy = paam_gen.generate("cfg4s", n_sys=n_search)
    b = pkg.paam_rta_load_systems(ctx, sy)
    r, _ = search_candidates(pkg, ctx, sy, b, "cfg4s")
    opts = pkg.analysis_opts()
    # the plain searches, each in the launch shape the search autotuner picks for it
    pkg.paam_rta_autotune_search(ctx, b, opts, r, stop_at_first=True)
    pkg.search(ctx, b, r, stop_at_first=True, want_cand_ok=False)
    t_ee, _ = _timed(lambda: pkg.search(ctx, b, r, stop_at_first=True, want_cand_ok=False), 3)
    pkg.paam_rta_autotune_search(ctx, b, opts, r)
    pkg.search(ctx, b, r)
    t_ex, (first_x, cand_x) = _timed(lambda: pkg.search(ctx, b, r), 3)
    S = sy.n_sys
    kx = min(1024, (16 * int(sy.chains_per_system().max()) + 63) // 64 * 64)  # the first layer's K
    order_k = torch.empty((S, top_k), dtype=torch.int32, device="cuda")
    order_all = torch.empty((S, K), dtype=torch.int32, device="cuda")
    first = torch.empty(S, dtype=torch.int32, device="cuda")
    cand = torch.empty((S, K), dtype=torch.uint8, device="cuda")

    def infer(order, pinned=SEARCH_PINNED):
        pkg.paam_surrogate_infer(ctx, model, b, r, order.shape[1], order, n_pinned=pinned)

    def guided(order, stop_at_first, cand_ok, pinned=SEARCH_PINNED):
        infer(order, pinned)
        pkg.paam_rta_search_ordered(ctx, b, opts, r, order, stop_at_first, cand_ok, first)
        return first

    # top-k: every one of the k best-scored candidates is confirmed exactly
    guided(order_k, False, cand)
    t_inf, _ = _timed(lambda: infer(order_k), 3)
    t_g, _ = _timed(lambda: guided(order_k, False, cand), 3)
    fx, cx = first_x.cpu().numpy(), cand_x.cpu().numpy().astype(bool)
    guided(order_k, False, cand)
    fg, cg = first.cpu().numpy(), cand.cpu().numpy().astype(bool)
    has = fx >= 0
    false_accepts = int(np.sum(cg & ~cx))
    recall = float((fg[has] >= 0).mean()) if has.any() else None
    # the network alone (no pinned seeds) under the same budget
    guided(order_k, False, cand, 0)
    recall_net = float((first.cpu().numpy()[has] >= 0).mean()) if has.any() else None
    # the same confirmation budget spent on the first k slots, and on k random slots
    slot_recall = float(cx[:, :top_k][has].any(axis=1).mean()) if has.any() else None
    rng = np.random.default_rng(3)
    pick = np.argsort(rng.random((S, K)), axis=1)[:, :top_k]
    rand_recall = float(np.take_along_axis(cx, pick, 1)[has].any(axis=1).mean()) if has.any() else None
    # exact verdicts (paam_surrogate_search): the pinned seeds of every system, then, for
    # the systems they do not admit, every other candidate in the network's order,
    # stopping at the first admitted one
    exact = lambda: pkg.paam_surrogate_search(ctx, model, b, opts, r, first, n_pinned=SEARCH_PINNED)
    exact()
    t_fb, _ = _timed(exact, 3)
    fb_first = first.cpu().numpy()
    fb_same = bool(np.array_equal(fb_first >= 0, has))
    fb_ok = bool(np.all(cx[np.nonzero(fb_first >= 0)[0], fb_first[fb_first >= 0]]))
    # recall of the network's own ranking (no pinned seeds) at other budgets
    infer(order_all, 0)
    ranked_all = order_all.cpu().numpy()
    ok_in_rank = np.take_along_axis(cx, ranked_all, 1)
    recall_at = {str(k): float(ok_in_rank[:, :k][has].any(axis=1).mean()) for k in (1, 2, 4, 8, 16, 32, 64)
                 if k <= K} if has.any() else {}
    b.free()
    model.free()
    return {
        "train": {"systems": rows, "sources": list(sources), "epochs": epochs, "lr": lr, "minibatch": 8192,
                  "label_analysis_s": round(t_label, 4), "train_s": round(t_train, 4),
                  "train_tflops": flops_train_row * rows * epochs / t_train / 1e12,
                  "train_flops_per_row": flops_train_row, "chunk_loss": losses,
                  "heldout_mae_R_over_D": mae},
        "workload": f"cfg4s: {S} systems x {K} candidate orders",
        "exhaustive_systems_per_s": S / t_ex, "exhaustive_ms": t_ex * 1e3,
        "early_exit_systems_per_s": S / t_ee, "early_exit_ms": t_ee * 1e3,
        "top_k": top_k, "pinned_seed_slots": SEARCH_PINNED,
        "guided_systems_per_s": S / t_g, "guided_ms": t_g * 1e3,
        "speedup_vs_exhaustive": t_ex / t_g, "speedup_vs_early_exit": t_ee / t_g,
        "infer_ms": t_inf * 1e3, "infer_tflops": fwd(kx) * S * K / t_inf / 1e12, "infer_flops_per_candidate": fwd(kx),
        "false_accepts": false_accepts, "recall": recall, "recall_network_only": recall_net,
        "recall_first_k_slots": slot_recall,
        "recall_random_k": rand_recall, "recall_at_k": recall_at,
        "fallback": {"method": "paam_surrogate_search: the pinned seeds, then the network's order for the systems "
                               "they do not admit, each system stopping at its first admitted candidate",
                     "systems_per_s": S / t_fb, "ms": t_fb * 1e3, "same_verdicts_as_exhaustive": fb_same,
                     "admitted_candidates_admissible": fb_ok,
                     "speedup_vs_exhaustive": t_ex / t_fb, "speedup_vs_early_exit": t_ee / t_fb},
    }


def gemm_bench(pkg, M, N, K, steps, warmup):
    """The network's tensor-core GEMM alone, fp32 output: TFLOP/s against the
    measured bf16 peak (first-layer shape of a 262,144-row inference chunk)."""
    import torch

    g = torch.Generator().manual_seed(5)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        pkg.paam_tc_gemm_bf16(A, B, C, err, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        pkg.paam_tc_gemm_bf16(A, B, C, err, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # spot check against a float32 product of the same bf16 operands
    rows = torch.arange(0, M, max(1, M // 64), device="cuda")
    ref = A[rows].float() @ B.float().t()
    rel = float(((C[rows] - ref).abs().max() / ref.abs().max()).item())
    tf = 2.0 * M * N * K / (ms / 1e3) / 1e12
    pk = peaks()
    return {"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "peak_tflops": pk["bf16_tflops"],
            "frac": tf / pk["bf16_tflops"], "peak_src": pk["src"], "max_rel_err_vs_fp32": rel,
            "err_flag": int(err.item())}


def end_to_end_bench(pkg, ctx, n_sys):
    """Chains spanning several executors (the workload's chains grouped into
    end-to-end chains of 1-3 sub-chains): the analysis of the sub-chains and
    the composition of their bounds."""
    import torch

    import paam_gen

    sy, off, chain, D = paam_gen.split_end_to_end(paam_gen.generate(WORKLOAD, n_sys=n_sys), 11)
    b = pkg.paam_rta_load_systems(ctx, sy)
    pkg.paam_rta_autotune(ctx, b, pkg.analysis_opts())
    R, st, _ = pkg.analyze(ctx, b)
    t = lambda a: torch.from_numpy(a).cuda()
    off_d, chain_d, D_d = t(off), t(chain), t(D)
    Re = torch.empty(len(D), dtype=torch.int64, device="cuda")
    se = torch.empty(len(D), dtype=torch.uint8, device="cuda")
    eps_prime = 198_000
    pkg.paam_rta_end_to_end(ctx, b, off_d, chain_d, D_d, eps_prime, R, st, Re, se)
    t_an, _ = _timed(lambda: pkg.analyze(ctx, b), 10)
    t_e2e, _ = _timed(lambda: pkg.paam_rta_end_to_end(ctx, b, off_d, chain_d, D_d, eps_prime, R, st, Re, se), 10)
    sts = se.cpu().numpy()
    b.free()
    return {"systems": sy.n_sys, "sub_chains": sy.n_chain, "end_to_end_chains": len(D),
            "eps_prime_ns": eps_prime, "analysis_ms": t_an * 1e3, "compose_ms": t_e2e * 1e3,
            "end_to_end_chains_per_s": len(D) / (t_an + t_e2e),
            "status_fractions": [float((sts == k).mean()) for k in range(3)]}


def kappa_bench(pkg, ctx, iters, sy=None):
    """The device preemption cost between the lowest and highest stream
    priority (the paper's method, four kernel kinds), and what the largest
    measured delay, used as kappa, does to the analysis with two buckets."""
    import torch

    out = {"iterations_per_kernel": iters}
    worst = 0.0
    for kind, name in enumerate(pkg.PREEMPTION_KERNELS):
        d, base = pkg.paam_measure_preemption(kind, iters)
        out[name] = {"mean_us": float(d.mean()), "max_us": float(d.max()), "stdev_us": float(d.std()),
                     "alone_us": float(np.median(base))}
        worst = max(worst, float(d.max()))
    kappa = int(round(worst * 1e3))
    out["kappa_ns"] = kappa
    if sy is not None:
        b = pkg.paam_rta_load_systems(ctx, sy)
        fr = {}
        for k in (0, kappa):
            R, st, v = pkg.analyze(ctx, b, n_buckets=2, kappa=k)
            torch.cuda.synchronize()
            fr[str(k)] = {"sched_chains": float((st == 0).float().mean().item()),
                          "sched_systems": float(v.float().mean().item())}
        b.free()
        out["analysis_n_buckets_2"] = fr
    return out


def accelerators_bench(pkg, ctx, n_sys, units=3):
    """The workload with its accelerator segments spread over `units` units by
    worst-fit decreasing (one server per unit, rule R1): analysed with
    per-accelerator tables (the register-table kernel up to four units)."""
    import torch

    import paam_gen

    base = paam_gen.generate(WORKLOAD, n_sys=n_sys)
    out = {"systems": n_sys, "units": units}
    for k, sy in (("1", base), (str(units), paam_gen.assign_accelerators(base, units))):
        b = pkg.paam_rta_load_systems(ctx, sy)
        pkg.paam_rta_autotune(ctx, b, pkg.analysis_opts())
        R, st, v = pkg.analyze(ctx, b)
        t, _ = _timed(lambda: pkg.analyze(ctx, b), 5)
        torch.cuda.synchronize()
        out[k] = {"ms": t * 1e3, "chains_per_s": sy.n_chain / t,
                  "sched_chains": float((st == 0).float().mean().item())}
        b.free()
    return out


def safe_blocking_bench(pkg, ctx, sy):
    """The same batch under the safe reading of Lemma 4's blocking term
    (blocking_mode 1: a lower-priority callback holds its executor for its
    WCET plus each of its segments' bounds), in the launch configuration the
    autotuner picks for that mode, beside the literal reading."""
    import torch

    b = pkg.paam_rta_load_systems(ctx, sy)
    out = {"systems": sy.n_sys}
    for mode, key in ((0, "literal"), (1, "safe")):
        opts = pkg.analysis_opts(blocking_mode=mode)
        pkg.paam_rta_autotune(ctx, b, opts)
        R, st, v = pkg.analyze(ctx, b, blocking_mode=mode)
        t, _ = _timed(lambda: pkg.analyze(ctx, b, blocking_mode=mode), 5)
        torch.cuda.synchronize()
        out[key] = {"ms": t * 1e3, "chains_per_s": sy.n_chain / t, "launch_config": pkg.paam_rta_get_launch_config(b),
                    "sched_chains": float((st == 0).float().mean().item())}
    b.free()
    return out


def infer_bench(pkg, n_sys, steps, warmup):
    """The network's ranking alone (features, 4 layers with the fused score,
    top-k) on the search workload, random weights: what a step of guided search
    spends before its exact confirmation."""
    import torch

    import paam_gen

    ctx = pkg.Context(0)
    rng = np.random.default_rng(1)
    sizes = [(1024, 256), (256, 256), (256, 256), (256, 64)]
    p = np.concatenate([np.concatenate([rng.uniform(-1, 1, fi * fo) * np.sqrt(6 / fi), rng.uniform(-.1, .1, fo)])
                        for fi, fo in sizes]).astype(np.float32)
    m = pkg.Model.create(ctx, 1)
    m.set_params(p)
    sy = paam_gen.generate("cfg4s", n_sys=n_sys)
    ranks = paam_gen.candidate_ranks(sy, SEARCH_K, paam_gen.CONFIGS["cfg4s"]["seed"] + 7)
    b = pkg.paam_rta_load_systems(ctx, sy)
    r = torch.from_numpy(ranks).cuda()
    ranked = torch.empty((n_sys, 16), dtype=torch.int32, device="cuda")
    for _ in range(warmup):
        pkg.paam_surrogate_infer(ctx, m, b, r, 16, ranked)
    t, _ = _timed(lambda: pkg.paam_surrogate_infer(ctx, m, b, r, 16, ranked), max(1, steps))
    b.free()
    m.free()
    return {"systems": n_sys, "candidates": n_sys * SEARCH_K, "ms": t * 1e3,
            "candidates_per_s": n_sys * SEARCH_K / t}


def search_cpu_baseline(pkg, ctx, n_sys):
    """The oracle's exhaustive search on the first n_sys systems of the
    sparse-executor search workload, and the GPU's exhaustive search on the
    same candidates compared with it (cand_ok and first_ok)."""
    import torch

    import oracle
    import paam_gen

    sy = paam_gen.generate("cfg4s", n_sys=n_sys)
    ranks = paam_gen.candidate_ranks(sy, SEARCH_K, paam_gen.CONFIGS["cfg4s"]["seed"] + 7)
    cores = os.cpu_count() or 1
    ranks[:, 0, :] = oracle.audsley(sy, nmax=ranks.shape[2], threads=cores)  # slot 0 as on the GPU, untimed
    t0 = time.perf_counter()
    ref = oracle.search(sy, ranks, threads=cores)
    dt = time.perf_counter() - t0
    b = pkg.paam_rta_load_systems(ctx, sy)
    first, cand = pkg.search(ctx, b, torch.from_numpy(ranks).cuda())
    same = bool(np.array_equal(first.cpu().numpy(), ref["first_ok"]) and
                np.array_equal(cand.cpu().numpy(), ref["cand_ok"]))
    b.free()
    return {"value": n_sys / dt, "unit": "systems/s (exhaustive, 256 candidates)", "cores": cores, "kind": "oracle",
            "sample": f"{n_sys} systems of the sparse-executor search workload", "bit_exact_vs_oracle": same}


# ---------------------------------------------------------------------------
# several ranks (one GPU each): shards by seed, slowest rank's time
# ---------------------------------------------------------------------------
def rank_seed(rank: int) -> int:
    """Seed of rank's own batch of the workload: each rank analyses different
    systems of the same shape (weak scaling, no data exchange)."""
    import paam_gen

    return paam_gen.CONFIGS[WORKLOAD]["seed"] + 1_000_003 * rank


def reduce_over_ranks(elapsed_ms: float, n_chain: int, n_sys: int, dist, device) -> tuple:
    """(slowest rank's time, chains and systems over all ranks); dist None on one rank."""
    import torch

    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([n_chain, n_sys], dtype=torch.int64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u[0].item()), int(u[1].item())


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    import paam_gen
    import paper_2404_06452_gb300 as pkg

    if args.gemm:
        if rank == 0:
            print(json.dumps({"gemm": gemm_bench(pkg, *args.gemm, args.steps, args.warmup)}), flush=True)
        return
    if args.infer:
        if rank == 0:
            print(json.dumps({"infer": infer_bench(pkg, args.infer, args.steps, args.warmup)}), flush=True)
        return
    if args.kappa:
        if rank == 0:
            print(json.dumps({"kappa": kappa_bench(pkg, pkg.Context(local), args.kappa)}), flush=True)
        return

    n_sys = args.n_sys or paam_gen.CONFIGS[WORKLOAD]["n_sys"]
    seed = rank_seed(rank)
    sy = paam_gen.generate(WORKLOAD, n_sys=n_sys, seed=seed)
    ctx = pkg.Context(local)
    stream = torch.cuda.Stream(device=local)
    batch = pkg.paam_rta_load_systems(ctx, sy, stream=stream)
    dev = torch.device("cuda", local)
    R = torch.empty(batch.n_chain, dtype=torch.int64, device=dev)
    st = torch.empty(batch.n_chain, dtype=torch.uint8, device=dev)
    verdict = torch.empty(batch.n_sys, dtype=torch.uint8, device=dev)
    opts = pkg.analysis_opts(1, 0, 0)
    # pick the launch configuration on this batch (untimed; results are identical for all)
    if args.launch_config is None:
        cfg_index, cfg_times = pkg.paam_rta_autotune(ctx, batch, opts, stream=stream)
    else:
        cfg_index, cfg_times = args.launch_config, []
        pkg.paam_rta_set_launch_config(batch, cfg_index)

    def step():
        pkg.paam_rta_analyze_batch(ctx, batch, opts, R, st, verdict, stream=stream)

    # ---- device-resident throughput ------------------------------------------
    sampler = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.launch_count() - launches0
    if dist:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    elapsed_ms, total_chains, total_sys = reduce_over_ranks(elapsed_ms, batch.n_chain, batch.n_sys, dist, dev)
    value = total_chains * args.steps / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / args.steps

    # ---- roofline of the dominant (only) kernel of the step ------------------
    pk = peaks()
    alg = algorithmic_bytes(sy)
    kern_ms = ms_per_step  # one analysis kernel per step
    achieved = alg / (kern_ms / 1e3) / 1e9
    traffic = traffic_per_system(WORKLOAD, cfg_index)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None if traffic is None else traffic * sy.n_sys,
                "traffic_src": "ncu capture of 500k systems, scaled per system" if traffic else None,
                "peak_src": pk["src"],
                "issue": None if WORKLOAD != "cfg2" or cfg_index not in WARP_INST_PER_SYSTEM else {
                    "bound": "issue", "unit": "warp-instructions/s",
                    "achieved": WARP_INST_PER_SYSTEM[cfg_index] * sy.n_sys / (kern_ms / 1e3),
                    "peak": ISSUE_PEAK,
                    "frac": WARP_INST_PER_SYSTEM[cfg_index] * sy.n_sys / (kern_ms / 1e3) / ISSUE_PEAK,
                    "note": "executed (not algorithmic) instructions per system, from the ncu capture"},
                "kernel": CONFIG_KERNEL.get(cfg_index, "analysis kernel"),
                "algorithmic_bytes_per_launch": alg}

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = None
    if rank == 0 or world > 1:
        pinned = pkg.to_device(sy, pin=True)
        hR = torch.empty(batch.n_chain, dtype=torch.int64).pin_memory()
        hst = torch.empty(batch.n_chain, dtype=torch.uint8).pin_memory()
        hv = torch.empty(batch.n_sys, dtype=torch.uint8).pin_memory()
        h2d = sum(getattr(pinned, f).numel() * getattr(pinned, f).element_size()
                  for f in ["sys_chain_off", "chain_cb_off", "cb_seg_off", "T", "D", "prio", "exec", "spin", "E",
                            "A", "acc", "sys_exec_off", "exec_core", "exec_prio"])
        d2h = hR.numel() * 8 + hst.numel() + hv.numel()

        def e2e_step():
            # one call: chunked host-to-device copies overlapped with validation,
            # analysis and the copies of R, status and verdict back to the host
            pkg.paam_rta_analyze_host(ctx, pinned, opts, hR, hst, hv, launch_config=cfg_index)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        dt = time.perf_counter() - t0
        dt_ms, e2e_chains, _ = reduce_over_ranks(dt * 1e3, batch.n_chain, batch.n_sys, dist, dev)
        dt = dt_ms / 1e3
        e2e = {"value": e2e_chains * args.e2e_steps / dt, "unit": "chains/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
               "ms_per_step": dt * 1e3 / args.e2e_steps}

    # ---- CPU baseline: the oracle on the host cores ---------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ref = oracle.analyze(sy, threads=cores)
        dt = time.perf_counter() - t0
        cpu = {"value": sy.n_chain / dt, "unit": "chains/s", "cores": cores, "kind": "oracle",
               "sample": f"the whole {sy.n_sys}-system workload, one pass", "cpu_model": cpu_model()}
        # one core, on a 50,000-system slice
        sl = sy.subset(np.arange(min(50_000, sy.n_sys)))
        t0 = time.perf_counter()
        oracle.analyze(sl, threads=1)
        cpu["single_core_value"] = sl.n_chain / (time.perf_counter() - t0)
        # the numbers above come from bit-identical results
        same = bool(np.array_equal(ref["R"], R.cpu().numpy()) and np.array_equal(ref["status"], st.cpu().numpy()))
        cpu["bit_exact_vs_gpu"] = same

    # ---- the other analysis workloads (single GPU, rank 0) ---------------------
    workloads = None
    if rank == 0 and world == 1 and not args.no_workloads:
        workloads = {cfg: workload_bench(pkg, ctx, cfg, args.workload_steps, max(3, args.warmup), 3,
                                         not args.no_cpu_baseline) for cfg in EXTRA_WORKLOADS if cfg != WORKLOAD}

    # ---- priority search and surrogate (single GPU, rank 0) -------------------
    search = surrogate = None
    if rank == 0 and world == 1 and not args.no_search:
        search = search_bench(pkg, ctx, args.search_sys)
        if not args.no_cpu_baseline:
            search["cpu_baseline"] = search_cpu_baseline(pkg, ctx, min(args.search_sys, 2000))
    if rank == 0 and world == 1 and not args.no_surrogate:
        surrogate = surrogate_bench(pkg, ctx, args.train_sys, args.search_sys, args.top_k)
    e2e_chains = kappa = accel = safe = None
    if rank == 0 and world == 1 and not args.no_search:
        e2e_chains = end_to_end_bench(pkg, ctx, min(n_sys, 1_000_000))
        accel = accelerators_bench(pkg, ctx, min(n_sys, 1_000_000))
        safe = safe_blocking_bench(pkg, ctx, sy if sy.n_sys <= 1_000_000 else sy.subset(np.arange(1_000_000)))
        if args.kappa_iters > 0:
            kappa = kappa_bench(pkg, ctx, args.kappa_iters, sy.subset(np.arange(min(sy.n_sys, 200_000))))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "chains/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "systems_per_gpu": batch.n_sys, "chains_per_gpu": batch.n_chain,
                       "l2": "inputs larger than L2 (%.2f GB per GPU)" % (sy.nbytes() / 1e9),
                       "parallelism": f"dp{world}" if world > 1 else "single GPU",
                       "launch_config": cfg_index,
                       "autotune_ms": [round(t, 4) for t in cfg_times]},
            "systems_per_s": total_sys * args.steps / (elapsed_ms / 1e3),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "search": search, "surrogate": surrogate, "end_to_end": e2e_chains, "kappa": kappa, "accelerators": accel,
            "safe_blocking": safe, "workloads": workloads,
        }
        print(json.dumps(line), flush=True)
    batch.free()
    if dist:
        dist.destroy_process_group()


def main():
    global WORKLOAD, WORKLOAD_DESC
    args = parse()
    if args.workload != WORKLOAD:
        WORKLOAD, WORKLOAD_DESC = args.workload, EXTRA_WORKLOADS[args.workload]["desc"]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
