"""Benchmark: E^H E applies/s of the CG reconstruction on the 2D 256x256, 32-coil,
35750-sample (71.5 ms) spiral with 3rd-order field terms.

One step = one sense_cg_solve: b = E^H s, then N_It = 40 CG iterations (each one E^H E
apply, the vector updates, the history row). value = N_It * steps / time (applies/s,
summed over ranks); the voxel*sample*coil rate is 2 L K C per apply.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
launching stream, with L2 flushed (a 256 MiB write) between steps; barrier + synchronize
around the timed region, max over ranks. The e2e figure calls the same public entry point
with HOST buffers (pinned): the H2D copy of Sigma and the D2H copy of the image are inside
its timed region. Clocks are sampled with nvidia-smi during the timed region.

--impl reference times the FP64 CPU oracle (the only other implementation of the method
here) on a bounded sample of the same workload, on the host cores.
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

METRIC = "E^H E applies/s (CG on the normal equations, on-the-fly encoding)"
UNIT = "applies/s"


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "tc_fp16", "tc_split"])
    ap.add_argument("--workload", default="target_256",
                    choices=["target_256", "precision_128", "plain_32", "stack_3d", "batch_64",
                             "batch_small_64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the (untimed) differentiation measurements")
    ap.add_argument("--no-stored", action="store_true",
                    help="skip the (untimed) stored-P comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the (untimed) 3D and batch workloads of the default line")
    ap.add_argument("--stored", action="store_true",
                    help="--op-only: stream stored phase tiles instead of generating them")
    ap.add_argument("--op-only", action="store_true",
                    help="time only W + K single E^H E applies (used for kernel profiling)")
    return ap.parse_args()


def run_op_only(args):
    """W warm-up and K timed sense_normal_op calls; prints one JSON line. The tensor-core
    E and E^H passes are the 2nd..(2K+1)th kernels after the warm-up ones."""
    import torch
    from paper_2604_09233_gb300 import native
    prec_name = "tc_split" if args.prec == "auto" else args.prec
    prec = native.PRECISIONS[prec_name]
    wl = _workload(args.workload)
    dev = torch.device("cuda", 0)
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    if args.stored:
        native.sense_plan_store_p(plan.handle, True)
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    out = torch.empty_like(m)
    for _ in range(args.warmup):
        native.sense_normal_op(plan.handle, prec, m, out)
    torch.cuda.synchronize()
    native.sense_plan_profile(plan.handle, True)
    for _ in range(args.steps):
        native.sense_normal_op(plan.handle, prec, m, out)
    torch.cuda.synchronize()
    st = native.sense_plan_stats(plan.handle)
    print(json.dumps({"op_only": True, "workload": wl.name, "precision": prec_name,
                      "stored": bool(args.stored),
                      "steps": args.steps, "stats": st}), flush=True)
    plan.close()


def _workload(name):
    from paper_2604_09233_gb300 import synthetic
    return getattr(synthetic, name)()


def _config(wl, prec_name):
    return {"workload": wl.name, "L": wl.L, "K": wl.K, "coils": wl.C, "basis_rows": wl.P1,
            "cg_iters": wl.n_iter, "precision": prec_name,
            "l2": "flushed between steps (256 MiB write)"}


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ------------------------------------------------------------------------------------------
def oracle_apply_rate(wl, budget_s=12.0):
    """Time the FP64 oracle's E and E^H on a sample of rows/voxels and extrapolate one
    E^H E apply linearly (both are sums over independent rows / voxels)."""
    import oracle
    rng = np.random.default_rng(0)
    m = wl.m_true
    y = wl.noise + 1.0
    n_rows, n_vox = 32, 32
    t0 = time.perf_counter()
    oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, j=wl.j, rows=np.arange(n_rows))
    t_enc = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, j=wl.j, vox=np.arange(n_vox))
    t_adj = time.perf_counter() - t0
    # grow the sample to use the budget
    scale = max(1.0, (budget_s / 2) / max(t_enc + t_adj, 1e-3))
    n_rows = int(min(wl.K, n_rows * scale))
    n_vox = int(min(wl.L, n_vox * scale))
    rows = np.sort(rng.choice(wl.K, n_rows, replace=False))
    vox = np.sort(rng.choice(wl.L, n_vox, replace=False))
    t0 = time.perf_counter()
    oracle.encode(wl.Kmat, wl.Rmat, wl.S, m, j=wl.j, rows=rows)
    t_enc = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.adjoint(wl.Kmat, wl.Rmat, wl.S, y, j=wl.j, vox=vox)
    t_adj = time.perf_counter() - t0
    t_apply = t_enc * wl.K / n_rows + t_adj * wl.L / n_vox
    return {"value": 1.0 / t_apply, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"E on {n_rows} of {wl.K} sample rows + E^H on {n_vox} of {wl.L} voxels, "
                      f"all coils, FP64, extrapolated linearly to one E^H E apply",
            "seconds": t_enc + t_adj}


def run_reference_batch(args):
    """Oracle on the batch mix: its voxel-sample-coil rate measured on a bounded sample of
    every 8th instance, converted to applies/s over the mix of all instances."""
    from paper_2604_09233_gb300 import synthetic
    wls = getattr(synthetic, args.workload)()
    per_step = max(2.0, 100.0 / max(1, args.steps + args.warmup))
    sample = wls[::8]

    def rate():
        # voxel*sample*coil products per second of the oracle (E and E^H)
        r = [oracle_apply_rate(w, budget_s=per_step / len(sample)) for w in sample]
        vsc = [2.0 * w.L * w.K * w.C * x["value"] for w, x in zip(sample, r)]
        return float(np.mean(vsc)), r[-1], sum(x["seconds"] for x in r)

    for _ in range(args.warmup):
        rate()
    vals, secs, last = [], 0.0, None
    for _ in range(args.steps):
        v, last, s = rate()
        secs += s
        vals.append(v)
    vsc_rate = float(np.mean(vals))
    t_mix = sum(2.0 * w.L * w.K * w.C for w in wls) / vsc_rate    # one apply of every instance
    value = len(wls) / t_mix
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOADS[args.workload], "instances": len(wls)},
        "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "value": value, "unit": UNIT,
                         "sample": f"E and E^H row/voxel samples of {len(sample)} of the "
                                   f"{len(wls)} instances, FP64, rate converted to the mix"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in BATCH_WORKLOADS:
        return run_reference_batch(args)
    wl = _workload(args.workload)
    per_step = max(2.0, 100.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_apply_rate(wl, budget_s=per_step)
    vals, secs = [], 0.0
    last = None
    for _ in range(args.steps):
        last = oracle_apply_rate(wl, budget_s=per_step)
        vals.append(last["value"])
        secs += last["seconds"]
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(wl, "fp64 oracle"),
        "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": value,
                                                                              "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
# DRAM bytes per launch of the tensor-core passes (dram__bytes_read.sum + dram__bytes_write.sum)
# and warp instructions executed per launch (smsp__inst_executed.sum), from one ncu capture of
# `python bench.py --op-only --steps 1 --warmup 2` (profiles/tcp_pass_2d256_32coil_sh3.md), keyed
# by the SHA-256 of the pass-kernel source they were taken on (pass_kernel_source_hash); any other
# source reports null.
KERNEL_TRAFFIC = {
    "6f4586b88a18f9ea82086326cf942c8d5ea6f378e416f2b19f8c856d6f945ea7": {
        "2d_256x256_32coil_35750samp_sh3": {
            "precision": "tc_split",
            "tc_encode_pass": 175048960 + 8707072,
            "tc_adjoint_pass": 169221376 + 10060288,
            "inst_tc_encode_pass": 1413535812,
            "inst_tc_adjoint_pass": 1413884787,
            # stored-P passes (the NKP = 0 instantiation of the same source): one capture of
            # `python bench.py --op-only --stored --steps 1 --warmup 1`
            # (profiles/tcp_pass_stored_2d256_32coil.md)
            "stored_tc_encode_pass": 19943396352 + 13079808,
            "stored_tc_adjoint_pass": 19573116928 + 17617920,
        },
    },
}


def pass_kernel_source_hash():
    """SHA-256 of the generated-tile pass kernel's code: sense_tcp.cu up to its launch helpers
    (the layout, the kernel and everything before it), then sense_ptx.cuh and sense_tc.cuh,
    with // comments and blank lines removed (they do not change the compiled kernel)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2604_09233_gb300", "csrc")

    def code(text):
        lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
        return "\n".join(ln for ln in lines if ln.strip()).encode()

    with open(os.path.join(csrc, "sense_tcp.cu")) as fh:
        text = fh.read()
    end = text.index("template <int MODE, int CP, int NPART, int NKP>\nstatic int launch(")
    h = hashlib.sha256(code(text[:end]))
    for name in ("sense_ptx.cuh", "sense_tc.cuh"):
        with open(os.path.join(csrc, name)) as fh:
            h.update(code(fh.read()))
    return h.hexdigest()


def _kernel_traffic(workload, prec_name, kernel):
    rec = KERNEL_TRAFFIC.get(pass_kernel_source_hash(), {}).get(workload)
    if not rec or rec["precision"] != prec_name:
        return None
    return rec.get(kernel)


GOLDEN_CG = {"2d_256x256_32coil_35750samp_sh3": os.path.join(ROOT, "tests", "golden",
                                                               "cg_target_256.txt")}


def golden_cg(workload):
    """FP64 oracle CG iterates stored for a workload (written by tests/golden/make_cg_target_256.py
    from the oracle alone): {"voxels": int array, "iterates": {n: complex array}} or None."""
    path = GOLDEN_CG.get(workload)
    if path is None or not os.path.exists(path):
        return None
    cols = None
    rows = []
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("# columns:"):
                cols = ln.split(":", 1)[1].split()
            elif ln.strip() and not ln.startswith("#"):
                rows.append([float(v) for v in ln.split()])
    a = np.asarray(rows)
    its = sorted({int(c.split("_")[1]) for c in cols[1:]})
    out = {"voxels": a[:, 0].astype(np.int64), "iterates": {}}
    for n in its:
        out["iterates"][n] = a[:, cols.index(f"re_{n}")] + 1j * a[:, cols.index(f"im_{n}")]
    return out


def max_over_ranks(total_ms, world, device=None):
    """The largest of the ranks' timed totals, returned on every rank (the job takes as long
    as its slowest replica)."""
    if world <= 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2604_09233_gb300 import native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec_name = "tc_split" if args.prec == "auto" else args.prec
    prec = native.PRECISIONS[prec_name]

    wl = _workload(args.workload)
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
    # coil data Sigma = E m + noise (E applied by the FP32 path; an input, not a result)
    s = plan.encode(m) + torch.from_numpy(wl.noise.astype(np.complex64)).to(dev)
    x = torch.empty(wl.L, dtype=torch.complex64, device=dev)
    n_it = wl.n_iter
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve(sv, xv, p=prec):
        native.sense_cg_solve(plan.handle, sv, xv, n_it, prec=p, history=False)

    for _ in range(max(3, args.warmup)):
        solve(s, x)
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    native.sense_plan_profile(plan.handle, True)
    times = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve(s, x)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    stats = native.sense_plan_stats(plan.handle)
    native.sense_plan_profile(plan.handle, False)
    if world > 1:
        dist.barrier()
    total_ms = max_over_ranks(float(np.sum(times)), world, dev)
    value = job_rate(n_it * args.steps, world, total_ms)
    x_tc = x.clone()

    # ---------------------------------------------------------------- comparisons (untimed)
    def apply_rate(p, reps=3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        native.sense_normal_op(plan.handle, p, m, x)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            native.sense_normal_op(plan.handle, p, m, x)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return reps / (ev[0].elapsed_time(ev[1]) / 1e3)

    rates = {name: apply_rate(native.PRECISIONS[name]) for name in ("fp32", "tc_fp16", "tc_split")}
    x_ref = torch.empty_like(x)
    native.sense_cg_solve(plan.handle, s, x_ref, n_it, prec=native.SENSE_PREC_FP32, history=False)
    torch.cuda.synchronize()
    err_vs_fp32 = (torch.linalg.norm(x_tc - x_ref) / torch.linalg.norm(x_ref)).item()

    # ---------------------------------------------------------------- vs the FP64 oracle (untimed)
    # relative L2 over the stored voxels of the CG iterates after n iterations, against the
    # FP64 oracle's CG (the CG loop of Alg. 1) on the same phantom and noise
    vs_oracle = None
    gold = golden_cg(wl.name)
    if gold is not None:
        vox = torch.from_numpy(gold["voxels"]).to(dev)
        vs_oracle = {"source": "tests/golden/cg_target_256.txt: FP64 oracle CG iterates on "
                               f"{len(gold['voxels'])} voxels (every 64th)",
                     "sigma": "E m by the FP32 path + the same noise; the oracle's own FP64 "
                              "E m differs by ~1e-7 relative, which CG amplifies with the "
                              "iteration count (FP64 CG moves by >1e-3 under such a "
                              "perturbation within 15-20 iterations)"}
        for name, pv in ((prec_name, prec), ("fp32", native.SENSE_PREC_FP32)):
            errs = {}
            for n_g, ref in gold["iterates"].items():
                if n_g == n_it and pv == prec:
                    xg = x_tc
                elif n_g == n_it and pv == native.SENSE_PREC_FP32:
                    xg = x_ref
                else:
                    xg = torch.empty_like(x)
                    native.sense_cg_solve(plan.handle, s, xg, n_g, prec=pv, history=False)
                got = xg[vox].cpu().numpy().astype(np.complex128)
                errs[str(n_g)] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            vs_oracle[name] = {"rel_l2_by_iterations": errs}

    # ---------------------------------------------------------------- e2e (host buffers)
    s_host = torch.empty((wl.K, wl.C), dtype=torch.complex64).pin_memory()
    s_host.copy_(s.cpu())
    x_host = torch.empty(wl.L, dtype=torch.complex64).pin_memory()
    e2e_t = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        native.sense_cg_solve(plan.handle, s_host.numpy(), x_host.numpy(), n_it, prec=prec,
                              history=False)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = job_rate(n_it * len(e2e_t), world,
                         max_over_ranks(1e3 * float(np.sum(e2e_t)), world, dev))

    # ---------------------------------------------------------------- differentiation (untimed)
    # 40-iteration CG with checkpoints every 8 iterations, its reverse pass (ds and d omega of
    # Re<w, x>), and the B0-gradient primitive of E (one t-weighted adjoint plus E^H g)
    diff = None
    if not args.no_grad:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        nbytes = native.sense_cg_ckpt_bytes(plan.handle, n_it, 8)
        ck = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        xg = torch.empty_like(x)
        sbar = torch.empty_like(s)
        wbar = torch.empty(wl.L, dtype=torch.float32, device=dev)
        xbar = torch.ones_like(x)
        native.sense_cg_solve_ckpt(plan.handle, s, xg, ck, n_it, 8, prec=prec)   # warm-up
        native.sense_cg_backward(plan.handle, s, ck, xbar, sbar=sbar, omega_bar=wbar)
        torch.cuda.synchronize()
        ev[0].record(stream)
        native.sense_cg_solve_ckpt(plan.handle, s, xg, ck, n_it, 8, prec=prec)
        ev[1].record(stream)
        native.sense_cg_backward(plan.handle, s, ck, xbar, sbar=sbar, omega_bar=wbar)
        ev[2].record(stream)
        gw = torch.empty(wl.L, dtype=torch.float32, device=dev)
        gz = torch.empty_like(x)
        native.sense_grad_b0(plan.handle, prec, m, s, gw, z=gz)
        ev[3].record(stream)
        native.sense_grad_b0(plan.handle, prec, m, s, gw, z=gz)
        ev[4].record(stream)
        torch.cuda.synchronize()
        fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        diff = {"cg_iters": n_it, "ckpt_every": 8, "forward_ms": fwd, "backward_ms": bwd,
                "backward_over_forward": bwd / fwd, "grad_b0_primitive_ms": ev[3].elapsed_time(ev[4]),
                "checkpoint_bytes": nbytes,
                "finite": bool(torch.isfinite(wbar).all().item() and torch.isfinite(sbar).all().item())}

    # ---------------------------------------------------------------- k-space filter (untimed)
    # the k-space filtering that ends Alg. 1 (Fig. 2), on the reconstructed image (2D workloads): convex-hull mask of the
    # first-order coefficients (host, once) and the filter (device)
    kfilter = None
    if len(wl.shape) == 2:
        N = wl.shape[0]
        d = wl.meta["fov"] / N
        cx = 1 if wl.Kmat.shape[1] == 3 else 2          # columns of (kx, ky) in K
        t0 = time.perf_counter()
        mask = native.sense_kspace_filter_mask(N, N, d, d, wl.Kmat[:, cx], wl.Kmat[:, cx + 1])
        t_mask = time.perf_counter() - t0
        mk = torch.from_numpy(mask.ravel()).to(dev)
        img = x_tc.clone()
        native.sense_kspace_filter(img, mk, wl.shape)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(3):
            native.sense_kspace_filter(img, mk, wl.shape)
        ev[1].record(stream)
        torch.cuda.synchronize()
        kfilter = {"filter_ms": ev[0].elapsed_time(ev[1]) / 3, "mask_host_ms": 1e3 * t_mask,
                   "mask_fraction": float(mask.mean())}

    # ---------------------------------------------------------------- stored P (untimed)
    # the paper's alternative: phase tiles computed once, streamed from HBM every pass
    stored = None
    if not args.no_stored:
        info_p = plan.info
        tile_bytes = 16 * info_p["L_padded"] * info_p["K_padded"]       # both passes, hi + lo
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        try:
            ev[0].record(stream)
            native.sense_plan_store_p(plan.handle, True)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_gen = ev[0].elapsed_time(ev[1])
            r_split = apply_rate(native.SENSE_PREC_TC_SPLIT, reps=5)
            r_fp16 = apply_rate(native.SENSE_PREC_TC_FP16, reps=5)
            x_st = torch.empty_like(x)
            native.sense_cg_solve(plan.handle, s, x_st, n_it, prec=prec, history=False)
            torch.cuda.synchronize()
            same = bool(torch.equal(x_st, x_tc)) if prec == native.SENSE_PREC_TC_SPLIT else None
            native.sense_plan_store_p(plan.handle, False)
            # per split apply the two passes read 8 bytes per (sample, voxel) pair each
            gbs = tile_bytes * r_split / 1e9
            stored = {"tile_bytes": tile_bytes, "generate_ms": t_gen,
                      "traffic_per_pass": {k: _kernel_traffic(wl.name, prec_name, "stored_" + k)
                                           for k in ("tc_encode_pass", "tc_adjoint_pass")},
                      "applies_per_s": {"tc_split": r_split, "tc_fp16": r_fp16},
                      "vs_generated": {"tc_split": r_split / rates["tc_split"],
                                       "tc_fp16": r_fp16 / rates["tc_fp16"]},
                      "tile_read_gbs_split": gbs,
                      "frac_of_measured_hbm": gbs / _peaks()[0]["hbm_gbs"],
                      "cg_bit_identical_to_generated": same}
        except native.SenseError as e:
            stored = {"unavailable": str(e)}

    # ---------------------------------------------------------------- map smoothing (untimed)
    # Eq. 1 on noisy copies of all coils' sensitivities (trusted mask M_T: the phantom's support,
    # |m| above 10 % of its peak; reconstruction mask M_R: M_T dilated by 8 voxels, so the maps
    # are extrapolated over an 8-voxel band; magnitude and normalised map of every coil, 2 C
    # fields in one solve) and Eq. 3 on a noisy B0 map (first differences weighted by a random
    # standard error), 2D workloads
    maps = None
    if len(wl.shape) == 2:
        from paper_2604_09233_gb300 import maps as smaps
        maps = {f"eq1_sensitivities_{wl.C}coil": smaps.run(wl, dilate=8)}
        rng = np.random.default_rng(8)
        n_vox = wl.L
        ones = np.ones(n_vox, np.float32)
        w = (wl.Rmat[0] + 20.0 * rng.normal(size=n_vox)).astype(np.complex64)
        eps = rng.uniform(0.2, 2.0, size=n_vox).astype(np.float32)
        dones, deps = torch.from_numpy(ones).to(dev), torch.from_numpy(eps).to(dev)
        dw = torch.from_numpy(w).to(dev)

        def timed(fn):
            fn()                                   # first call untimed
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            res = fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]), res

        maps["eq3_b0"] = {"fields": 1}
        for pc in ("multigrid", "none"):
            out = torch.empty_like(dw)
            ms, inf = timed(lambda: native.sense_smooth_map(
                wl.shape, 1, 2.0, dones, deps, dw, out, max_iter=20000, rel_tol=1e-6,
                precond=pc))
            maps["eq3_b0"][pc] = {"ms": ms, "iterations": inf["iters"],
                                  "rel_residual": inf["rel_residual"]}

    # ---------------------------------------------------------------- 3D and batch (untimed)
    # the other named workloads, measured on the same GPU in the same run: the 3D stack of
    # spirals (applies/s of E^H E per precision and a few CG iterations against the FP32
    # path) and both 64-instance batches (one batched solve each against the same instances
    # solved one after another)
    extra3d, batches = None, None
    if not args.no_extra and args.workload == "target_256" and world == 1:
        extra3d = measure_3d(dev, prec_name)
        batches = {}
        for bw in BATCH_WORKLOADS:
            try:
                r = batch_measure(bw, prec_name, 1, 1, dev, full=False)
                batches[bw] = {k: r[k] for k in ("value", "ms_per_step", "speedup_vs_sequential",
                                                 "sequential_single_problem_ms",
                                                 "voxel_sample_coil_gops", "roofline",
                                                 "iterations_per_instance")}
                batches[bw]["unit"] = UNIT + " summed over instances"
                batches[bw]["config"] = r["config"]
            except native.SenseError as e:
                batches[bw] = {"unavailable": str(e)}

    # ---------------------------------------------------------------- roofline
    # dominant kernel: the tensor-core pass (E or E^H) with the larger share of event time
    peaks, peak_kind = _peaks()
    sincos_peak = native.sense_diag_sincos_rate(300.0)
    info = plan.info
    Lp, Kp, Cp = info["L_padded"], info["K_padded"], info["C_padded"]
    kc = "tc_encode_pass" if stats["tc_encode_pass"]["ms"] >= stats["tc_adjoint_pass"]["ms"] \
        else "tc_adjoint_pass"
    n_launch = max(1, stats[kc]["n"])
    t_launch = stats[kc]["ms"] / n_launch / 1e3
    pairs = float(Lp) * float(Kp)                  # phase pairs generated per launch
    achieved_sincos = pairs / t_launch
    mma_per_pair = 6 if prec_name == "tc_split" else 2
    flops = pairs * mma_per_pair * 2 * (2 * Cp)    # 2 * N per pair per MMA, N = 2 Cp
    tflops = flops / t_launch / 1e12
    peak_tc = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    traffic = _kernel_traffic(wl.name, prec_name, kc)
    sfu = {"bound": "alu", "achieved": achieved_sincos / 1e9, "peak": sincos_peak / 1e9,
           "unit": "Gsincos/s", "frac": achieved_sincos / sincos_peak, "traffic": traffic,
           "kernel": kc, "per_launch_ms": t_launch * 1e3,
           "peak_source": "measured on this GPU by sense_diag_sincos_rate"}
    tensor = {"bound": "tensor", "achieved": tflops, "peak": peak_tc, "unit": "TFLOP/s",
              "frac": tflops / peak_tc, "traffic": traffic, "kernel": kc,
              "peak_source": f"bf16 sustained, {peak_kind} (fp16 = bf16 rate)"}
    roof = sfu if sfu["frac"] >= tensor["frac"] else tensor
    # the pass is bound by instruction issue in its generator warps: warp instructions per
    # second against one per clock per SM sub-partition
    clocks = clk.summary()
    inst = _kernel_traffic(wl.name, prec_name, "inst_" + kc)
    issue = None
    if inst is not None:
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_issue = 4.0 * n_sm * mhz * 1e6
        issue = {"bound": "issue", "achieved": inst / t_launch / 1e9,
                 "peak": peak_issue / 1e9, "unit": "Gwarp-inst/s",
                 "frac": inst / t_launch / peak_issue, "kernel": kc, "inst_per_launch": inst,
                 "peak_source": "4 warp instructions per clock per SM at the median sampled SM "
                                "clock; instructions per launch from ncu for this kernel code"}

    vsc = 2.0 * wl.L * wl.K * wl.C
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16" if prec != 0 else "f32",
        "data": "synthetic", "config": _config(wl, prec_name),
        "voxel_sample_coil_gops": value * vsc / 1e9,
        "applies_per_s_by_precision": rates,
        "speedup_vs_fp32_path": rates["tc_split"] / rates["fp32"],
        "cg_rel_err_vs_fp32_path": err_vs_fp32,
        "cg_vs_fp64_oracle": vs_oracle,
        "roofline": roof,
        "roofline_other": tensor if roof is sfu else sfu,
        "roofline_issue": issue,
        "kernel_ms": {k: stats[k]["ms"] for k in native.KERNEL_CLASSES},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": wl.K * wl.C * 8,
                "d2h_bytes_per_step": wl.L * 8},
        "gpu_launches": stats["launches"],
    }
    if diff is not None:
        line["differentiation"] = diff
    if kfilter is not None:
        line["kspace_filter"] = kfilter
    if stored is not None:
        line["stored_p"] = stored
    if maps is not None:
        line["map_smoothing"] = maps
    if extra3d is not None:
        line["stack_3d"] = extra3d
    if batches is not None:
        line["batch"] = batches
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_apply_rate(wl)
        cb.pop("seconds")
        # the same oracle on one host core (a smaller sample)
        import oracle
        n_threads = oracle.num_threads()
        oracle.set_num_threads(1)
        try:
            one = oracle_apply_rate(wl, budget_s=4.0)
        finally:
            oracle.set_num_threads(n_threads)
        cb["single_core"] = {"value": one["value"], "unit": UNIT, "cores": 1,
                             "sample": one["sample"]}
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def measure_3d(dev, prec_name, cg_iters=5):
    """The 3D workload (96x96x48, 32 coils, 48 x 1300 samples, 2nd-order terms), untimed
    within the benchmark step: E^H E applies/s per precision (three applies each, events on
    the launching stream) and a short CG in the benchmark precision against the FP32 path."""
    import torch
    from paper_2604_09233_gb300 import native, synthetic
    wl = synthetic.stack_3d()
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    plan = native.Plan(wl.Kmat, wl.Rmat, wl.S, wl.j)
    t_plan = time.perf_counter() - t0
    try:
        m = torch.from_numpy(wl.m_true.astype(np.complex64)).to(dev)
        s = plan.encode(m) + torch.from_numpy(wl.noise.astype(np.complex64)).to(dev)
        q = torch.empty_like(m)

        def rate(p, reps):
            native.sense_normal_op(plan.handle, p, m, q)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(reps):
                native.sense_normal_op(plan.handle, p, m, q)
            ev[1].record(stream)
            torch.cuda.synchronize()
            return reps / (ev[0].elapsed_time(ev[1]) / 1e3)

        rates = {"tc_split": rate(native.SENSE_PREC_TC_SPLIT, 3),
                 "tc_fp16": rate(native.SENSE_PREC_TC_FP16, 3),
                 "fp32": rate(native.SENSE_PREC_FP32, 2)}
        prec = native.PRECISIONS[prec_name]
        x = torch.empty_like(m)
        xr = torch.empty_like(m)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        native.sense_cg_solve(plan.handle, s, x, cg_iters, prec=prec, history=False)
        ev[1].record(stream)
        native.sense_cg_solve(plan.handle, s, xr, cg_iters, prec=native.SENSE_PREC_FP32,
                              history=False)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(x - xr) / torch.linalg.norm(xr)).item()
        info = plan.info
        return {"workload": wl.name, "L": wl.L, "K": wl.K, "coils": wl.C,
                "applies_per_s_by_precision": rates,
                "speedup_vs_fp32_path": rates["tc_split"] / rates["fp32"],
                "voxel_sample_coil_gops_split": rates["tc_split"] * 2.0 * wl.L * wl.K * wl.C / 1e9,
                "cg_iters": cg_iters, "cg_ms": ev[0].elapsed_time(ev[1]),
                "cg_rel_err_vs_fp32_path": err, "plan_create_s": t_plan,
                "padded": [info["L_padded"], info["K_padded"], info["C_padded"]]}
    finally:
        plan.close()


BATCH_METRIC = "E^H E applies/s summed over instances (batched CG, uneven instances)"


BATCH_WORKLOADS = {"batch_64": "batch_64_2d_uneven", "batch_small_64": "batch_64_2d_small"}


def batch_measure(workload, prec_name, steps, warmup, dev, full=True):
    """64 independent uneven 2D instances solved by one batched CG (per-instance stop at
    relative residual 1e-3, at most 50 iterations). A step is one sense_batch_cg_solve.
    batch_64: matrices {64..256}^2 (most instances fill the GPU alone); batch_small_64:
    matrices {64, 96}^2 with 4096-8192 samples, where one instance underfills 152 SMs.
    Returns the measured fields; full=False skips the clock sampling and the e2e leg."""
    import torch
    from paper_2604_09233_gb300 import native, synthetic
    prec = native.PRECISIONS[prec_name]
    wls = getattr(synthetic, workload)()
    t0 = time.perf_counter()
    batch = native.Batch([(w.Kmat, w.Rmat, w.S, w.j) for w in wls])
    t_create = time.perf_counter() - t0
    tune = native.sense_batch_autotune(batch.handle, prec)
    n_it, tol = 50, 1e-3
    sig = []
    for i, w in enumerate(wls):
        plan = native.sense_batch_plan(batch.handle, i)
        enc = torch.empty((w.K, w.C), dtype=torch.complex64, device=dev)
        native.sense_encode(plan, native.SENSE_PREC_FP32,
                            torch.from_numpy(w.m_true.astype(np.complex64)).to(dev), enc)
        sig.append(enc + torch.from_numpy(w.noise.astype(np.complex64)).to(dev))
    xs = [torch.empty(w.L, dtype=torch.complex64, device=dev) for w in wls]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def solve():
        return native.sense_batch_cg_solve(batch.handle, sig, xs, n_it, prec=prec, rel_tol=tol)

    for _ in range(max(1, warmup)):
        infos = solve()
    torch.cuda.synchronize()
    times = []
    clk = ClockSampler(dev.index) if full else None
    if clk is not None:
        clk.__enter__()
    try:
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    finally:
        if clk is not None:
            clk.__exit__(None, None, None)
    total_ms = float(np.sum(times))
    iters = [inf["iters"] for inf in infos]
    applies = float(sum(iters))
    value = applies * steps / (total_ms / 1e3)
    vsc = sum(it * 2.0 * w.L * w.K * w.C for it, w in zip(iters, wls))

    # the same instances solved one after another through the single-problem API
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for i, w in enumerate(wls):
        native.sense_cg_solve(native.sense_batch_plan(batch.handle, i), sig[i], xs[i], n_it,
                              prec=prec, rel_tol=tol, history=False)
    ev[1].record(stream)
    torch.cuda.synchronize()
    seq_ms = ev[0].elapsed_time(ev[1])

    # roofline of the batched E^H E (both persistent passes and the per-instance kernels),
    # timed by the autotuner: phase pairs generated per apply / time
    pairs = 0.0
    for i in range(len(wls)):
        inf = native.sense_plan_info(native.sense_batch_plan(batch.handle, i))
        pairs += 2.0 * inf["L_padded"] * inf["K_padded"]
    sincos_peak = native.sense_diag_sincos_rate(300.0)
    achieved = pairs / (tune["ms"] / 1e3)
    n = len(wls)
    out = {
        "value": value, "ms_per_step": total_ms / steps,
        "config": {"workload": BATCH_WORKLOADS[workload], "instances": n,
                   "matrices": sorted({w.shape[0] for w in wls}),
                   "coils": sorted({w.C for w in wls}),
                   "samples": [min(w.K for w in wls), max(w.K for w in wls)],
                   "max_iter": n_it, "rel_tol": tol, "precision": prec_name,
                   "l2": "flushed between steps (256 MiB write)"},
        "voxel_sample_coil_gops": vsc * steps / (total_ms / 1e3) / 1e9,
        "iterations_per_instance": iters,
        "sequential_single_problem_ms": seq_ms,
        "speedup_vs_sequential": seq_ms / (total_ms / steps),
        "autotune": tune,
        "batch_create_s": t_create,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": sincos_peak / 1e9,
                     "unit": "Gsincos/s", "frac": achieved / sincos_peak, "traffic": None,
                     "kernel": "batched E^H E (two persistent passes + per-instance kernels)",
                     "peak_source": "measured on this GPU by sense_diag_sincos_rate"},
        # per step: 8 kernels per instance outside the loop (data layout, ||s||, E^H s: 4,
        # CG init, result) + per iteration 2 batched passes + 8 per instance
        "gpu_launches": 8 * n + n_it * (2 + 8 * n),
    }
    if full:
        out["clocks"] = clk.summary()
        # e2e: pinned host data in, solve, images out
        s_host = [sv.cpu().pin_memory() for sv in sig]
        x_host = [torch.empty(w.L, dtype=torch.complex64).pin_memory() for w in wls]
        e2e_t = []
        for i in range(steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for d, h in zip(sig, s_host):
                d.copy_(h, non_blocking=True)
            solve()
            for h, d in zip(x_host, xs):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t1)
        out["e2e"] = {"value": applies * len(e2e_t) / float(np.sum(e2e_t)), "unit": UNIT,
                      "h2d_bytes_per_step": int(sum(w.K * w.C * 8 for w in wls)),
                      "d2h_bytes_per_step": int(sum(w.L * 8 for w in wls))}
    batch.close()
    return out


def run_batch(args):
    """The batch workloads as the benchmark's own line (see batch_measure)."""
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prec_name = "tc_split" if args.prec == "auto" else args.prec
    res = batch_measure(args.workload, prec_name, args.steps, max(3, args.warmup), dev)
    line = {"metric": BATCH_METRIC, "value": res.pop("value"), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
            "data": "synthetic", "config": res.pop("config")}
    line.update(res)
    print(json.dumps(line), flush=True)


def main():
    args = _parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.op_only:
        run_op_only(args)
    elif args.workload in BATCH_WORKLOADS:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
