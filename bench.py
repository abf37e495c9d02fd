"""Throughput of the exact modular GEMM hot path on GB300.

Default workload: C <- C - (P A Q) * B mod 65521 with n = 8192 (M = N = K),
uint32 residues, i.i.d. uniform. One step is one pass of the whole path:
row-major A, B, C (resident in HBM) -> Morton-hybrid (T' = 128) with TURBO's
row/column permutations applied to A -> balanced int8 limb split -> tcgen05
limb GEMM with the exact mod-p recombine/subtract epilogue -> C back to
row-major. The plain CUDA-core form (aligned/contained decomposition of
Sec. 2.2, T' = 64) and the FP64 DFMA form run the same step for comparison.

value     = 2 M N K / (device time of one step), Gop/s (algorithmic ops only)
e2e       = same, through host buffers: pinned H2D of A, B, C and D2H of C
            inside the timed region, as 16-bit residues for p < 2^16 (the
            library's _u16 layout calls; the 32-bit transfer is reported in
            e2e.u32)
roofline  = the limb GEMM kernel: tensor work 2 M N K x (limb products: 3
            with Karatsuba on w = 2 limbs) per launch / its CUDA-event
            duration, against the measured bf16 burst peak (f16 runs at the
            bf16 rate; the kernel runs 2 ms at a time between lighter
            launches); traffic = its ncu DRAM bytes per launch
gf2       = C += A*B over GF(2) on bit-packed Morton-hybrid matrices (the
            paper's experimental field; E4M3 tensor cores), and the paper's
            workload of 468 random sub-matrix products in 2048 x 2048 matrices
configs   = the other workloads: 256^3 (launch-latency bound, next to the floor of
            one launch), the 3000 x 1700 x 2200 Schur update with permuted
            conversion, and 4096^3 at p = 2^31 - 1 on the limb form
curves    = Morton-hybrid against Hilbert-hybrid tile order: layout conversion
            and the permutation gather (index conversion per entry)

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fm|reference]
For N > 1 launch with torchrun; every rank runs an independent replica.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact modular GEMM Gop/s (2MNK/s) at p=65521, n=8192: INT8-limb vs plain, 1 GB300"
P = 65521
N_DEFAULT = 8192


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fm", choices=["fm", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip plain / DFMA comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-GEMM measurement")
    ap.add_argument("--no-tu", action="store_true", help="skip the TU decomposition measurement")
    ap.add_argument("--no-gf2", action="store_true", help="skip the GF(2) measurements")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the small, Schur-update and 31-bit workloads")
    ap.add_argument("--case", default=None,
                    choices=["gemm", "gemm_p31", "gemm_plain", "permute", "to_morton_permuted", "tu", "batch"],
                    help="profiling aid: run one kernel's call --steps times at --n (T' = --T) after "
                         "--warmup calls, print nothing else, exit")
    ap.add_argument("--T", type=int, default=128, help="T' of the --case matrices")
    ap.add_argument("--calls", type=int, default=4096, help="calls of the --case batch workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_setup(args, backend=None):
    """One process per GPU under torchrun (RANK, LOCAL_RANK, WORLD_SIZE and
    MASTER_* from the environment): NCCL on the GPUs, or `backend` (gloo on
    host cores) when given. The ranks are independent replicas; the group only
    carries the barriers and the max over ranks of the timed region."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend in (None, "nccl"):
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ops_per_step, steps, max_ms, world):
    """Whole-job throughput in Gop/s: every rank runs `steps` steps of
    `ops_per_step` operations; the job takes the slowest rank's time."""
    return world * ops_per_step * steps / (max_ms / 1e3) / 1e9


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        load = [s for s in sm if mx and s > 0.5 * mx] or sm
        med = load[len(load) // 2] if load else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), d.get("hbm_gbs"), "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


def profiled_traffic(kernel_src: str, name: str, n: int):
    """DRAM bytes per launch of a kernel at size n, from a committed ncu figure
    (profiles/<name>, JSON: source_sha256, n, traffic_bytes_per_launch), if the
    kernel's source has not changed since it was taken and it was taken at n."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    if rec.get("source_sha256") != sha or int(rec.get("n", -1)) != n:
        return None
    v = rec.get("traffic_bytes_per_launch")
    return float(v) if v is not None else None


# ---------------------------------------------------------------------------
def cpu_oracle_rate(n, p, target_s, threads=0):
    """Times the oracle's C - A*B mod p on a bounded sample of rows of the
    n x n x n product (host cores). Returns (Gop/s, cores, sample text, seconds)."""
    import fm_inputs
    import oracle
    cores = oracle.set_threads(threads)
    B = fm_inputs.uniform_residues(7, (n, n), p, 2)
    A = fm_inputs.uniform_residues(7, (n, n), p, 1)
    C = fm_inputs.uniform_residues(7, (n, n), p, 3)
    rows = min(n, 2 * cores)
    t0 = time.perf_counter()
    oracle.gemm_modp(C[:rows], A[:rows], B, p, oracle.OP_SUB)
    dt = time.perf_counter() - t0
    rows = max(rows, min(n, int(rows * target_s / max(dt, 1e-3)) // cores * cores))
    t0 = time.perf_counter()
    oracle.gemm_modp(C[:rows], A[:rows], B, p, oracle.OP_SUB)
    dt = time.perf_counter() - t0
    ops = 2.0 * rows * n * n
    return ops / dt / 1e9, cores, f"{rows} rows of C - A*B mod {p}, n={n} (K=N=n)", dt


def run_reference(args, world, rank):
    """The oracle (plain CPU triple loop) as the reference arm."""
    if rank != 0:
        return
    import numpy as np

    import fm_inputs
    import oracle
    n = args.n
    cores = oracle.set_threads(0)
    B = fm_inputs.uniform_residues(7, (n, n), P, 2)
    # size one step to ~1/ (steps + warmup) of a ~3 minute budget
    probe_rows = cores
    A = fm_inputs.uniform_residues(7, (probe_rows, n), P, 1)
    C = fm_inputs.uniform_residues(7, (probe_rows, n), P, 3)
    t0 = time.perf_counter()
    oracle.gemm_modp(C, A, B, P, oracle.OP_SUB)
    dt = time.perf_counter() - t0
    per_step_budget = 150.0 / max(1, args.steps + args.warmup)
    rows = max(1, min(n, int(probe_rows * per_step_budget / max(dt, 1e-3))))
    A = fm_inputs.uniform_residues(7, (rows, n), P, 1)
    C = fm_inputs.uniform_residues(7, (rows, n), P, 3)
    for _ in range(args.warmup):
        oracle.gemm_modp(C, A, B, P, oracle.OP_SUB)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.gemm_modp(C, A, B, P, oracle.OP_SUB)
    total = time.perf_counter() - t0
    ops = 2.0 * rows * n * n
    value = ops * args.steps / total / 1e9
    sample = f"{rows} rows of C - A*B mod {P} per step, n={n} (K=N=n)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gop/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64 accumulate (u128), mod p", "data": "synthetic",
        "config": {"workload": f"C -= A*B mod {P}, n={n}, row-major, CPU oracle", "n": n, "p": P},
        "cpu_baseline": {"value": value, "unit": "Gop/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_batched(fm, torch, dev, stream, args, count=4096, lo=32, hi=512, seed=5):
    """The batching form: count independent calls C_c -= A_c * B_c mod p with
    M, N, K uniform in [lo, hi], each on its own cell of a large Morton C and
    on random rectangles of shared Morton A and B. The workload is laid out at
    T' = 32, 64 and 128; at each T' the autotuner (fm_autotune_batch) times the
    plan forms on the batch and an FM_ALGO_AUTO plan takes the fastest; the
    fastest T' is the tuned choice. At T' = 64 the fixed forms are timed as
    well: the tensor-core limb plan (3 launches), the fused limb plan (1
    launch), the decomposed plain plan (1 persistent launch) and one
    fm_gemm_modp launch per call; every result is checked equal to the
    tuned plan's. The roofline is HBM: each call's A, B and C read and C
    written once."""
    import numpy as np

    import fm_inputs
    p = P
    big = 16384
    rows, cells = fm_inputs.batch_workload(seed, count, lo, hi, big)
    nC = cells * hi
    A = torch.from_numpy(fm_inputs.uniform_residues(seed, (big, big), p, 1).view(np.int32)).to(dev)
    B = torch.from_numpy(fm_inputs.uniform_residues(seed, (big, big), p, 2).view(np.int32)).to(dev)
    ops = 0.0
    algo_bytes = 0.0  # each call reads A, B and C and writes C once (4-byte residues)
    for c in range(count):
        M, N, K = (int(x) for x in rows[c, :3])
        algo_bytes += 4.0 * (M * K + K * N + 2 * M * N)
        ops += 2.0 * M * N * K
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3

    def timed(run):
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def layout(lt):
        tA = torch.empty(big * big, dtype=torch.int32, device=dev)
        tB = torch.empty_like(tA)
        mA = fm.matrix(tA, (big >> lt).bit_length() - 1, lt)
        mB = fm.matrix(tB, (big >> lt).bit_length() - 1, lt)
        fm.fm_layout_to_morton(A, big, big, big, mA)
        fm.fm_layout_to_morton(B, big, big, big, mB)
        tC = torch.zeros(nC * nC, dtype=torch.int32, device=dev)
        mC = fm.matrix(tC, (nC >> lt).bit_length() - 1, lt)
        calls = []
        for c in range(count):
            M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rows[c])
            call = fm.fm_gemm_call()
            call.C, call.A, call.B = fm.sub(mC, rC, cC, M, N), fm.sub(mA, rA, cA, M, K), fm.sub(mB, rB, cB, K, N)
            call.op = fm.FM_OP_SUB
            calls.append(call)
        return (tA, tB, tC), calls

    def form_name(r):
        if r.algo == fm.FM_ALGO_PLAIN:
            return "decomposed plain plan (1 persistent launch)"
        o = r.opts
        if o.fused_batch:
            return "fused limb plan (1 launch)"
        return (f"limb plan with planes (3 launches), tile width {o.block_n or 'default'}, K chunk "
                f"{o.k_chunk or 'full'}, {'no ' if o.no_karatsuba else ''}Karatsuba")

    fm.fm_autotune_clear()
    by_T = {}
    best = None
    for lt in (5, 6, 7):
        bufs, calls = layout(lt)
        r = fm.fm_autotune_batch(calls, p, 0, stream)
        plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_AUTO)
        ms = timed(lambda: plan.run(stream))
        by_T[f"T'={1 << lt}"] = {"form": form_name(r), "ms": ms, "value": ops / (ms / 1e3) / 1e9,
                                 "launches": plan.launches, "candidates": r.candidates,
                                 "tuner_ms": r.ms}
        if best is None or ms < best[1]:
            best = (lt, ms, plan.launches, form_name(r))
        plan.close()
        del bufs, calls
        torch.cuda.empty_cache()
    tuned_lt, tuned_ms, tuned_launches, tuned_form = best

    # the tuned choice again from scratch (its result is the reference below),
    # then the fixed forms at T' = 64 on the same inputs
    bufs, calls = layout(tuned_lt)
    plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_AUTO)
    plan.run(stream)
    torch.cuda.synchronize()
    tuned_out = torch.empty((nC, nC), dtype=torch.int32, device=dev)
    fm.fm_layout_from_morton(fm.matrix(bufs[2], (nC >> tuned_lt).bit_length() - 1, tuned_lt), nC, nC, tuned_out,
                             nC, stream)
    plan.close()
    del bufs, calls
    bufs, calls = layout(6)
    tC = bufs[2]
    mC = fm.matrix(tC, (nC >> 6).bit_length() - 1, 6)
    snap = tC.clone()
    check = torch.empty_like(tuned_out)

    def same_as_tuned():
        torch.cuda.synchronize()
        fm.fm_layout_from_morton(mC, nC, nC, check, nC, stream)
        torch.cuda.synchronize()
        return bool(torch.equal(check, tuned_out))

    fixed = {}
    for name, algo, o in (("limb", fm.FM_ALGO_LIMB_TC, None), ("fused", fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1)),
                          ("plain", fm.FM_ALGO_PLAIN, None)):
        pl = fm.fm_plan_create(calls, p, algo, o)
        tC.copy_(snap)
        pl.run(stream)
        same = same_as_tuned()
        ms = timed(lambda: pl.run(stream))
        fixed[name] = {"ms": ms, "value": ops / (ms / 1e3) / 1e9, "launches": pl.launches,
                       "output_tiles_or_items": pl.work_items, "bit_identical_to_tuned": same}
        pl.close()
    tC.copy_(snap)
    for call in calls:  # one launch per call, from the same state
        fm.fm_gemm_modp(call.C, call.A, call.B, p, call.op, fm.FM_ALGO_PLAIN, None, stream)
    per_call_same = same_as_tuned()
    per_call_ms = timed(lambda: [fm.fm_gemm_modp(c_.C, c_.A, c_.B, p, c_.op, fm.FM_ALGO_PLAIN, None, stream)
                                 for c_ in calls])
    del bufs, calls, snap, check, tuned_out, A, B
    torch.cuda.empty_cache()
    _, _, hbm_peak, peak_src = measured_peaks()
    ach = algo_bytes / (tuned_ms / 1e3) / 1e9
    return {"workload": f"{count} calls C -= A*B mod {p}, M,N,K ~ U[{lo},{hi}], Morton-hybrid, T' and plan form "
                        "chosen by the autotuner",
            "value": ops / (tuned_ms / 1e3) / 1e9, "unit": "Gop/s", "ms": tuned_ms, "launches": tuned_launches,
            "tuned": {"T": 1 << tuned_lt, "form": tuned_form, "by_T": by_T},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                         "per_call_frac": algo_bytes / (per_call_ms / 1e3) / 1e9 / hbm_peak,
                         "work": "algorithmic bytes: A, B, C read and C written once per call, 4 B each "
                                 f"({algo_bytes / 1e9:.3f} GB)", "peak_source": f"HBM copy, {peak_src}"},
            "per_call_ms": per_call_ms, "per_call_value": ops / (per_call_ms / 1e3) / 1e9,
            "speedup_vs_per_call": per_call_ms / tuned_ms, "per_call_launches": count,
            "per_call_bit_identical_to_tuned": per_call_same,
            "fixed_forms_at_T64": fixed}


def run_tu(fm, torch, dev, stream, m=16384, n=12288, k=10000, seed=5):
    """The TU decomposition workload: rank-revealing PLUQ over GF(65521) of an
    m x n matrix built as the product of seeded uniform m x k and k x n factors
    (rank k). Every trailing update is one fm_gemm_modp call. Timed once after
    one warm-up factorisation of the same matrix."""
    import numpy as np

    import fm_inputs
    p = P
    lt = 7

    def grid(r, c):
        lg = 0
        while (1 << lg) << lt < max(r, c):
            lg += 1
        return lg

    def morton_from(x):
        g = grid(*x.shape)
        side = (1 << g) << lt
        t = torch.zeros(side * side, dtype=torch.int32, device=dev)
        mm = fm.matrix(t, g, lt)
        src = torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(dev)
        fm.fm_layout_to_morton(src, x.shape[0], x.shape[1], x.shape[1], mm, stream)
        return t, mm

    tX, mX = morton_from(fm_inputs.uniform_residues(seed, (m, k), p, 1))
    tY, mY = morton_from(fm_inputs.uniform_residues(seed, (k, n), p, 2))
    g = grid(m, n)
    side = (1 << g) << lt
    tA = torch.zeros(side * side, dtype=torch.int32, device=dev)
    mA = fm.matrix(tA, g, lt)
    fm.fm_gemm_modp(fm.sub(mA, 0, 0, m, n), fm.sub(mX, 0, 0, m, k), fm.sub(mY, 0, 0, k, n), p,
                    fm.FM_OP_SET, fm.FM_ALGO_LIMB_TC, None, stream)
    del tX, tY
    orig = tA.clone()
    rp = torch.zeros(m, dtype=torch.int32, device=dev)
    cp = torch.zeros(n, dtype=torch.int32, device=dev)
    fm.fm_pluq(mA, m, n, p, rp, cp, stream)  # warm-up
    tA.copy_(orig)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fm.fm_pluq(mA, m, n, p, rp, cp, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ops = 2.0 * (m * n * r - (m + n) * r * r / 2.0 + r ** 3 / 3.0)
    del tA, orig
    return {"workload": f"rank-revealing PLUQ over GF({p}) of {m}x{n}, rank {k} (product of "
                        f"seeded uniform factors), 128-column panels, trailing updates via fm_gemm_modp",
            "ms": ms, "rank": r, "rank_expected": k, "value": ops / (ms / 1e3) / 1e9, "unit": "Gop/s",
            "ops": "2*(m n r - (m+n) r^2/2 + r^3/3)"}


def run_configs(fm, torch, dev, stream, peaks, seed=21):
    """The other workloads of the hot path, each timed with CUDA events after
    warm-up, and each result checked bit-identical against a second GEMM form
    on the same inputs:
    small   -- C = A*B mod 65521 at 256^3, T' = 32, plain form: a launch-latency
               bound call, reported in microseconds next to the floor of one
               launch of the library's smallest kernel (a 1 x 1 validation scan);
               checked against the limb form;
    schur   -- C (3000 x 2200) -= A (3000 x 1700) * B (1700 x 2200) mod 65521,
               T' = 64, row-major inputs converted on the device with random row
               and column permutations of A, plain form (aligned/contained
               decomposition); checked against the limb form;
    p31     -- C = A*B mod 2^31 - 1 at 4096^3, limb form (four limbs, 10 limb
               products on the tensor cores: Karatsuba over every pair of
               limbs); checked against the plain form."""
    import numpy as np

    import fm_inputs
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    s = stream.cuda_stream
    out = {}

    def dev_i32(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(dev)

    def morton(side, lt):
        lg = 0
        while (1 << lg) << lt < side:
            lg += 1
        n_ = (1 << lg) << lt
        t = torch.zeros(n_ * n_, dtype=torch.int32, device=dev)
        return t, fm.matrix(t, lg, lt)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def same_as(tC, snap, run_other):
        # the result in tC against the other form run on the same inputs
        got = tC.clone()
        tC.copy_(snap)
        run_other()
        torch.cuda.synchronize()
        return bool(torch.equal(tC, got))

    # small: 256^3, plain, T' = 32
    p = 65521
    n = 256
    A = fm_inputs.uniform_residues(seed, (n, n), p, 1)
    B = fm_inputs.uniform_residues(seed, (n, n), p, 2)
    (tA, mA), (tB, mB), (tC, mC) = morton(n, 5), morton(n, 5), morton(n, 5)
    fm.fm_layout_to_morton(dev_i32(A), n, n, n, mA, s)
    fm.fm_layout_to_morton(dev_i32(B), n, n, n, mB, s)
    sub = [fm.sub(m_, 0, 0, n, n) for m_ in (mC, mA, mB)]

    def small(algo):
        fm.fm_gemm_modp(sub[0], sub[1], sub[2], p, fm.FM_OP_SET, algo, None, s)

    us = timed(lambda: small(fm.FM_ALGO_PLAIN), 200) * 1e3
    one = fm.sub(mA, 0, 0, 1, 1)
    floor_us = timed(lambda: fm.fm_validate_residues(one, p, s), 200) * 1e3
    # where the time of a call goes: host submission (200 calls queued without
    # waiting), and the device alone (the call replayed from a CUDA graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(200):
        small(fm.FM_ALGO_PLAIN)
    host_us = (time.perf_counter() - t0) / 200 * 1e6
    torch.cuda.synchronize()
    gs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        fm.fm_gemm_modp(sub[0], sub[1], sub[2], p, fm.FM_OP_SET, fm.FM_ALGO_PLAIN, None, gs.cuda_stream)
    graph_us = timed(lambda: graph.replay(), 200) * 1e3
    del graph
    torch.cuda.synchronize()
    same = same_as(tC, tC.clone(), lambda: small(fm.FM_ALGO_LIMB_TC))
    out["small"] = {"workload": "C = A*B mod 65521, M=N=K=256, Morton-hybrid T'=32, plain form",
                    "us_per_call": us, "launch_floor_us": floor_us, "floor_frac": floor_us / us,
                    "host_submit_us_per_call": host_us, "graph_replay_us_per_call": graph_us,
                    "value": 2.0 * n ** 3 / (us / 1e6) / 1e9, "unit": "Gop/s", "bit_identical_to_limb": same}
    del tA, tB, tC

    # schur: 3000 x 1700 x 2200 with permutations, plain, T' = 64
    M, K, N = 3000, 1700, 2200
    dA = dev_i32(fm_inputs.uniform_residues(seed, (M, K), p, 3))
    dB = dev_i32(fm_inputs.uniform_residues(seed, (K, N), p, 4))
    dC = dev_i32(fm_inputs.uniform_residues(seed, (M, N), p, 5))
    drp, dcp = dev_i32(fm_inputs.permutation(seed, M, 6)), dev_i32(fm_inputs.permutation(seed, K, 7))
    side = max(M, K, N)  # one common 2^m T' grid (4096 x 4096 at T' = 64)
    (tA, mA), (tB, mB), (tC, mC) = morton(side, 6), morton(side, 6), morton(side, 6)
    sC, sA, sB = fm.sub(mC, 0, 0, M, N), fm.sub(mA, 0, 0, M, K), fm.sub(mB, 0, 0, K, N)

    def layout():
        fm.fm_layout_to_morton_permuted(dA, M, K, K, drp, dcp, mA, s)
        fm.fm_layout_to_morton(dB, K, N, N, mB, s)
        fm.fm_layout_to_morton(dC, M, N, N, mC, s)

    lay_ms = timed(layout, 10)
    gemm_ms = timed(lambda: fm.fm_gemm_modp(sC, sA, sB, p, fm.FM_OP_SUB, fm.FM_ALGO_PLAIN, None, s), 5)
    layout()
    snap = tC.clone()
    fm.fm_gemm_modp(sC, sA, sB, p, fm.FM_OP_SUB, fm.FM_ALGO_PLAIN, None, s)
    torch.cuda.synchronize()
    same = same_as(tC, snap, lambda: fm.fm_gemm_modp(sC, sA, sB, p, fm.FM_OP_SUB, fm.FM_ALGO_LIMB_TC, None, s))
    ops = 2.0 * M * N * K
    lay_bytes = 8.0 * (M * K + K * N + M * N)
    out["schur"] = {"workload": "C(3000x2200) -= A(3000x1700) * B(1700x2200) mod 65521, Morton-hybrid T'=64, "
                                "row and column permutations of A in the conversion, plain form",
                    "layout_ms": lay_ms, "layout_gbs": lay_bytes / (lay_ms / 1e3) / 1e9, "gemm_ms": gemm_ms,
                    "value": ops / (gemm_ms / 1e3) / 1e9, "unit": "Gop/s", "bit_identical_to_limb": same,
                    "gemm_frac_of_imad_wide": (ops / 2 / (gemm_ms / 1e3) / 1e12 / peaks["imad_wide"]
                                               if peaks else None)}
    del tA, tB, tC, dA, dB, dC, snap

    # p31: 4096^3 at p = 2^31 - 1, limb form (T' = 128); the plain form, which
    # takes T' = 32 or 64, computes the same product on T' = 64 copies
    p = 2147483647
    n = 4096
    xa = dev_i32(fm_inputs.uniform_residues(seed, (n, n), p, 10))
    xb = dev_i32(fm_inputs.uniform_residues(seed, (n, n), p, 11))
    res = []
    for lt, algo in ((7, fm.FM_ALGO_LIMB_TC), (6, fm.FM_ALGO_PLAIN)):
        (tA, mA), (tB, mB), (tC, mC) = morton(n, lt), morton(n, lt), morton(n, lt)
        fm.fm_layout_to_morton(xa, n, n, n, mA, s)
        fm.fm_layout_to_morton(xb, n, n, n, mB, s)
        sub = [fm.sub(m_, 0, 0, n, n) for m_ in (mC, mA, mB)]
        run = lambda: fm.fm_gemm_modp(sub[0], sub[1], sub[2], p, fm.FM_OP_SET, algo, None, s)  # noqa: E731
        if algo == fm.FM_ALGO_LIMB_TC:
            ms = timed(run, 5)
        else:
            run()
        o = torch.empty((n, n), dtype=torch.int32, device=dev)
        fm.fm_layout_from_morton(mC, n, n, o, n, s)
        res.append(o)
        del tA, tB, tC
    torch.cuda.synchronize()
    same = bool(torch.equal(res[0], res[1]))
    del xa, xb, res
    burst, _, _, src = measured_peaks()
    # four limbs, Karatsuba over every pair: 4 + 6 = 10 limb products
    mma = 10 * 2.0 * n ** 3 / (ms / 1e3) / 1e12
    out["p31"] = {"workload": "C = A*B mod 2^31-1, M=N=K=4096, Morton-hybrid T'=128, limb form (4 limbs, "
                              "10 limb products: Karatsuba over every pair of limbs)", "ms": ms,
                  "value": 2.0 * n ** 3 / (ms / 1e3) / 1e9,
                  "ceiling_gops": 1e3 * burst / 10, "frac_of_ceiling": 2.0 * n ** 3 / (ms / 1e3) / 1e9 / (1e3 * burst / 10),
                  "unit": "Gop/s", "mma_tflops": mma, "frac_of_tensor_peak": mma / burst,
                  "peak_source": f"bf16 burst, {src}", "bit_identical_to_plain": same}
    torch.cuda.empty_cache()
    return out


def run_curves(fm, torch, dev, stream, n=8192, seed=31):
    """The curve comparison of Sec. 1 on this GPU: layout conversion (one index
    conversion per tile) and the row/column permutation gather (one index
    conversion per entry) at n x n, for the Morton-hybrid and the Hilbert-hybrid
    layouts, at T' = 32 and 128. Rates are bytes moved (4 B read + 4 B written
    per entry) per second; the two curves' results are checked to hold the same
    matrix."""
    import numpy as np

    import fm_inputs
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    s = stream.cuda_stream
    x = torch.from_numpy(fm_inputs.uniform_residues(seed, (n, n), 65521).view(np.int32)).to(dev)
    rp = torch.from_numpy(fm_inputs.permutation(seed, n, 1).view(np.int32)).to(dev)
    cp = torch.from_numpy(fm_inputs.permutation(seed, n, 2).view(np.int32)).to(dev)
    buf = [torch.empty(n * n, dtype=torch.int32, device=dev) for _ in range(2)]
    scratch = torch.empty((n, n), dtype=torch.int32, device=dev)
    permuted = {k: torch.empty((n, n), dtype=torch.int32, device=dev) for k in ("morton", "hilbert")}
    gbs = lambda ms: 8.0 * n * n / (ms / 1e3) / 1e9  # noqa: E731

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    for lt in (5, 7):
        lg = (n >> lt).bit_length() - 1
        m0, m1 = fm.matrix(buf[0], lg, lt), fm.matrix(buf[1], lg, lt)
        row = {}
        for name, to_, from_, perm in (
                ("morton", fm.fm_layout_to_morton, fm.fm_layout_from_morton, fm.fm_permute_rows_cols),
                ("hilbert", fm.fm_layout_to_hilbert, fm.fm_layout_from_hilbert, fm.fm_permute_rows_cols_hilbert)):
            t_to = timed(lambda: to_(x, n, n, n, m0, s))
            t_from = timed(lambda: from_(m0, n, n, scratch, n, s))
            t_perm = timed(lambda: perm(m0, m1, n, n, rp, cp, s))
            from_(m1, n, n, permuted[name], n, s)
            row[name] = {"to_layout_gbs": gbs(t_to), "from_layout_gbs": gbs(t_from),
                         "permute_gbs": gbs(t_perm), "permute_ms": t_perm}
        torch.cuda.synchronize()
        row["same_permuted_matrix"] = bool(torch.equal(permuted["morton"], permuted["hilbert"]))
        row["hilbert_over_morton_permute_time"] = row["hilbert"]["permute_ms"] / row["morton"]["permute_ms"]
        res[f"T'={1 << lt}"] = row
    del x, rp, cp, buf, scratch, permuted
    torch.cuda.empty_cache()
    return {"workload": f"{n} x {n} residues: row-major <-> curve layout, and the row/column "
                        "permutation gather inside the layout", "unit": "GB/s", "by_T": res}


def run_gf2(fm, torch, dev, stream, n=8192, paper_n=2048, paper_calls=468, seed=7):
    """GF(2) on bit-packed Morton-hybrid matrices (T' = 32): C += A*B at n, checked
    bit-identical to the uint32 limb form at p = 2 on the same inputs, then timed
    (3 warm-up + 10 timed calls, CUDA events); and the experiments' workload,
    paper_calls products of random sub-matrices of paper_n x paper_n matrices,
    timed back to back after one warm-up pass."""
    import numpy as np

    import fm_inputs
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    lg = 0
    while (32 << lg) < n:
        lg += 1
    words = (32 << lg) ** 2 // 32

    def packed(x):
        t = torch.zeros(words, dtype=torch.int32, device=dev)
        m = fm.gf2_matrix(t, lg)
        src = torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(dev)
        fm.fm_gf2_pack(src, n, n, n, m, stream)
        return t, m, src

    tA, mA, sA = packed(fm_inputs.uniform_residues(seed, (n, n), 2, 1))
    tB, mB, sB = packed(fm_inputs.uniform_residues(seed, (n, n), 2, 2))
    tC, mC, sC = packed(fm_inputs.uniform_residues(seed, (n, n), 2, 3))
    C, A, B = fm.gf2_sub(mC, 0, 0, n, n), fm.gf2_sub(mA, 0, 0, n, n), fm.gf2_sub(mB, 0, 0, n, n)
    # the same product through the uint32 limb form at p = 2
    lt = 7
    lgm = 0
    while (1 << lgm) << lt < n:
        lgm += 1
    side = (1 << lgm) << lt
    mats = []
    for src in (sA, sB, sC):
        t = torch.zeros(side * side, dtype=torch.int32, device=dev)
        mm = fm.matrix(t, lgm, lt)
        fm.fm_layout_to_morton(src, n, n, n, mm, stream)
        mats.append((t, mm))
    fm.fm_gemm_modp(fm.sub(mats[2][1], 0, 0, n, n), fm.sub(mats[0][1], 0, 0, n, n),
                    fm.sub(mats[1][1], 0, 0, n, n), 2, fm.FM_OP_ADD, fm.FM_ALGO_LIMB_TC, None, stream)
    limb_out = torch.empty(n * n, dtype=torch.int32, device=dev)
    fm.fm_layout_from_morton(mats[2][1], n, n, limb_out, n, stream)
    fm.fm_gf2_gemm(C, A, B, fm.FM_OP_ADD, None, stream)
    gf2_out = torch.empty(n * n, dtype=torch.int32, device=dev)
    fm.fm_gf2_unpack(mC, n, n, gf2_out, n, stream)
    torch.cuda.synchronize()
    identical = bool(torch.equal(limb_out, gf2_out))
    del mats, limb_out, gf2_out
    for _ in range(3):
        fm.fm_gf2_gemm(C, A, B, fm.FM_OP_ADD, None, stream)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        fm.fm_gf2_gemm(C, A, B, fm.FM_OP_ADD, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    e0.record(stream)
    for _ in range(10):
        fm.fm_gf2_pack(sC, n, n, n, mC, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pack = e0.elapsed_time(e1) / 10
    status = fm.fm_get_last_device_status(stream)
    del tA, tB, tC, sA, sB, sC
    # the experiments' workload: random sub-matrix products in paper_n x paper_n
    # matrices; every product is its own experiment, so each writes its own C
    # matrix (random C rectangles of one matrix would overlap)
    plg = 0
    while (32 << plg) < paper_n:
        plg += 1
    pw = (32 << plg) ** 2 // 32
    pm = []
    for q in range(3):
        t = torch.zeros(pw, dtype=torch.int32, device=dev)
        src = torch.from_numpy(fm_inputs.uniform_residues(seed + 1, (paper_n, paper_n), 2, q)
                               .view(np.int32)).to(dev)
        fm.fm_gf2_pack(src, paper_n, paper_n, paper_n, fm.gf2_matrix(t, plg), stream)
        pm.append((t, fm.gf2_matrix(t, plg)))
    rects = fm_inputs.sub_rectangles(seed, paper_calls, paper_n)
    cs = pm[0][0].repeat(paper_calls)  # paper_calls copies of the first matrix
    cmats = [fm.gf2_matrix(cs[c * pw:(c + 1) * pw], plg) for c in range(paper_calls)]
    calls = [(fm.gf2_sub(cmats[c], int(r[3]), int(r[4]), int(r[0]), int(r[1])),
              fm.gf2_sub(pm[1][1], int(r[5]), int(r[6]), int(r[0]), int(r[2])),
              fm.gf2_sub(pm[2][1], int(r[7]), int(r[8]), int(r[2]), int(r[1]))) for c, r in enumerate(rects)]
    ops = float(sum(2.0 * int(r[0]) * int(r[1]) * int(r[2]) for r in rects))
    snap = cs.clone()
    for c in calls:
        fm.fm_gf2_gemm(*c, fm.FM_OP_ADD, None, stream)
    torch.cuda.synchronize()
    per_call_result = cs.clone()
    e0.record(stream)
    for c in calls:
        fm.fm_gf2_gemm(*c, fm.FM_OP_ADD, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1)
    # the same products as one plan: three launches for the whole batch
    gcalls = []
    for c in calls:
        g = fm.fm_gf2_call()
        g.C, g.A, g.B = c
        g.op = fm.FM_OP_ADD
        gcalls.append(g)
    plan = fm.fm_gf2_plan_create(gcalls)
    cs.copy_(snap)
    plan.run(stream)
    torch.cuda.synchronize()
    plan_same = bool(torch.equal(cs, per_call_result))
    for _ in range(2):
        plan.run(stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        plan.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plan_ms = e0.elapsed_time(e1) / 5
    plan.close()
    del pm, cs, snap, per_call_result
    return {"workload": f"C += A*B over GF(2), n={n}, bit-packed Morton-hybrid T'=32, E4M3 tensor cores",
            "value": 2.0 * n ** 3 / (ms / 1e3) / 1e9, "unit": "Gop/s", "ms": ms, "pack_ms": ms_pack,
            "bit_identical_to_limb_p2": identical, "status": status,
            "paper_workload": {"workload": f"{paper_calls} products of random sub-matrices of "
                                           f"{paper_n}x{paper_n} bit-packed Morton-hybrid matrices, T'=32 "
                                           f"(one C matrix per product)",
                               "ms": pms, "value": ops / (pms / 1e3) / 1e9, "unit": "Gop/s",
                               "mean_call_us": pms * 1e3 / paper_calls,
                               "plan": {"ms": plan_ms, "value": ops / (plan_ms / 1e3) / 1e9,
                                        "unit": "Gop/s", "launches": 3,
                                        "speedup_vs_per_call": pms / plan_ms,
                                        "bit_identical_to_per_call": plan_same}}}


def run_fm(args, world, rank, local):
    import numpy as np
    import torch

    import fm_inputs
    import paper_1705_04807_gb300 as fm
    from paper_1705_04807_gb300 import build as fmbuild

    if rank == 0 or world == 1:
        fmbuild.build()
    barrier(world)
    fm.lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    n = args.n
    p = P
    w = 2
    lt_limb, lt_plain = 7, 6

    def lg_for(lt):
        lg = 0
        while (1 << lg) << lt < n:
            lg += 1
        return lg

    # seeded host inputs (same on every rank: replicas)
    A = fm_inputs.uniform_residues(1, (n, n), p, 1)
    B = fm_inputs.uniform_residues(1, (n, n), p, 2)
    C = fm_inputs.uniform_residues(1, (n, n), p, 3)
    rp = fm_inputs.permutation(1, n, 4)
    cp = fm_inputs.permutation(1, n, 5)

    def dev_i32(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(dev)

    dA, dB, dC = dev_i32(A), dev_i32(B), dev_i32(C)
    drp, dcp = dev_i32(rp), dev_i32(cp)
    dOut = torch.empty((n, n), dtype=torch.int32, device=dev)

    def morton(lt):
        lg = lg_for(lt)
        side = (1 << lg) << lt
        t = torch.empty(side * side, dtype=torch.int32, device=dev)
        return t, fm.matrix(t, lg, lt)

    tA, mA = morton(lt_limb)
    tB, mB = morton(lt_limb)
    tC, mC = morton(lt_limb)
    sA, sB, sC = fm.sub(mA, 0, 0, n, n), fm.sub(mB, 0, 0, n, n), fm.sub(mC, 0, 0, n, n)
    pa = torch.empty(fm.fm_limb_planes_size(n, n, fm.FM_LIMB_A, p) // 4 + 4, dtype=torch.int32,
                     device=dev)
    pb = torch.empty(fm.fm_limb_planes_size(n, n, fm.FM_LIMB_B, p) // 4 + 4, dtype=torch.int32,
                     device=dev)
    s = stream.cuda_stream

    def layout_in(srcA, srcB, srcC, mA_, mB_, mC_, u16=False):
        if u16:  # 16-bit row-major residues (p < 2^16)
            fm.fm_layout_to_morton_permuted_u16(srcA, n, n, n, drp, dcp, mA_, s)
            fm.fm_layout_to_morton_u16(srcB, n, n, n, mB_, s)
            fm.fm_layout_to_morton_u16(srcC, n, n, n, mC_, s)
        else:
            fm.fm_layout_to_morton_permuted(srcA, n, n, n, drp, dcp, mA_, s)
            fm.fm_layout_to_morton(srcB, n, n, n, mB_, s)
            fm.fm_layout_to_morton(srcC, n, n, n, mC_, s)

    kern = {"layout_in": [], "limb_split": [], "limb_gemm": [], "layout_out": []}

    def limb_step(srcA=dA, srcB=dB, srcC=dC, out=dOut, ev=None, u16=False):
        if ev:
            ev[0].record(stream)
        layout_in(srcA, srcB, srcC, mA, mB, mC, u16)
        if ev:
            ev[1].record(stream)
        fm.fm_limb_split(sA, fm.FM_LIMB_A, p, pa, None, s)
        fm.fm_limb_split(sB, fm.FM_LIMB_B, p, pb, None, s)
        if ev:
            ev[2].record(stream)
        fm.fm_limb_gemm(sC, pa, pb, n, p, fm.FM_OP_SUB, None, s)
        if ev:
            ev[3].record(stream)
        if u16:
            fm.fm_layout_from_morton_u16(mC, n, n, out, n, s)
        else:
            fm.fm_layout_from_morton(mC, n, n, out, n, s)
        if ev:
            ev[4].record(stream)

    launches_per_step = 3 + 2 + 1 + 1

    # ---- device-timed region (inputs resident in HBM, 3 x 256 MiB > L2) ----
    for _ in range(args.warmup):
        limb_step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        limb_step(ev=evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    for ev in evs:
        kern["layout_in"].append(ev[0].elapsed_time(ev[1]))
        kern["limb_split"].append(ev[1].elapsed_time(ev[2]))
        kern["limb_gemm"].append(ev[2].elapsed_time(ev[3]))
        kern["layout_out"].append(ev[3].elapsed_time(ev[4]))
    local_ms = t_start.elapsed_time(t_end)
    total_ms = allreduce_max(local_ms, world)
    ops = 2.0 * n * n * n
    value = job_value(ops, args.steps, total_ms, world)
    st = fm.fm_get_last_device_status(s)
    assert st == 0, f"device status {st}"

    # ---- end to end through host buffers ----
    # Every step copies its inputs from pinned host memory and reads its result
    # back. Steps are pipelined: the host-to-device copies of step k+1 and the
    # device-to-host copy of step k-1 run on their own streams while step k
    # computes (double-buffered device inputs and outputs). Residues mod
    # p < 2^16 travel as 16-bit entries (the library's _u16 layout calls), half
    # the bytes of the 32-bit form, which is measured as well.
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e(u16):
        hdt, ddt = (np.uint16, torch.int16) if u16 else (np.uint32, torch.int32)
        view = np.int16 if u16 else np.int32
        hA, hB, hC = (torch.from_numpy(x.astype(hdt).view(view)).pin_memory() for x in (A, B, C))
        hOut = [torch.empty((n, n), dtype=ddt).pin_memory() for _ in range(2)]
        xin = [tuple(torch.empty((n, n), dtype=ddt, device=dev) for _ in range(3)) for _ in range(2)]
        xout = [torch.empty((n, n), dtype=ddt, device=dev) for _ in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_comp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def steps_(count):
            for k in range(count):
                b = k & 1
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(ev_comp[b])    # step k-2 no longer reads these buffers
                    for dst, src in zip(xin[b], (hA, hB, hC)):
                        dst.copy_(src, non_blocking=True)
                    ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                if k >= 2:
                    stream.wait_event(ev_out[b])       # step k-2's result has left xout[b]
                limb_step(xin[b][0], xin[b][1], xin[b][2], xout[b], u16=u16)
                ev_comp[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_comp[b])
                    hOut[b].copy_(xout[b], non_blocking=True)
                    ev_out[b].record(s_out)
            stream.wait_stream(s_out)
            stream.wait_stream(s_in)

        steps_(2)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        steps_(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = allreduce_max(e0.elapsed_time(e1), world)
        # the results read back equal the device-resident result
        last = hOut[(args.steps - 1) & 1]
        want = dOut.cpu()
        same = bool(torch.equal(last.to(torch.int32) & 0xFFFF, want) if u16 else torch.equal(last, want))
        assert same
        esz = 2 if u16 else 4
        return {"value": job_value(ops, args.steps, ms, world), "unit": "Gop/s",
                "h2d_bytes_per_step": 3 * n * n * esz, "d2h_bytes_per_step": n * n * esz,
                "host_dtype": "u16" if u16 else "u32", "ms_per_step": ms / args.steps}

    e2e_u32 = e2e(False)
    if p < (1 << 16):
        e2e_line = e2e(True)
        e2e_line["u32"] = e2e_u32
    else:
        e2e_line = e2e_u32

    # ---- measured arithmetic rates of the non-tensor pipes (T multiply-adds/s) ----
    # (with the comparison forms only: the plain and DFMA rooflines use them)
    peaks = {} if args.no_compare else {name: fm.fm_measure_peak(kind, 1 << 16, s) / 1e12 for name, kind in (
        ("imad_wide", fm.FM_PEAK_IMAD_WIDE), ("imad32", fm.FM_PEAK_IMAD32), ("dfma", fm.FM_PEAK_DFMA),
        ("ffma", fm.FM_PEAK_FFMA), ("mma_s8", fm.FM_PEAK_MMA_S8))}

    out = {}
    # ---- comparison forms on the same inputs (same step, other GEMM) ----
    if not args.no_compare:
        tA6, mA6 = morton(lt_plain)
        tB6, mB6 = morton(lt_plain)
        tC6, mC6 = morton(lt_plain)
        s6 = [fm.sub(m_, 0, 0, n, n) for m_ in (mC6, mA6, mB6)]

        def plain_step(algo, ev=None):
            layout_in(dA, dB, dC, mA6, mB6, mC6)
            if ev:
                ev[0].record(stream)
            fm.fm_gemm_modp(s6[0], s6[1], s6[2], p, fm.FM_OP_SUB, algo, None, s)
            if ev:
                ev[1].record(stream)
            fm.fm_layout_from_morton(mC6, n, n, dOut, n, s)

        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        limb_step()
        torch.cuda.synchronize()
        ref = dOut.clone()
        for name, algo, steps, kind in (("plain", fm.FM_ALGO_PLAIN, 3, "imad_wide"),
                                        ("dfma", fm.FM_ALGO_DFMA, 1, "dfma")):
            plain_step(algo)
            torch.cuda.synchronize()
            gev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
            e0.record(stream)
            for k in range(steps):
                plain_step(algo, gev[k])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            gemm_ms = sum(g[0].elapsed_time(g[1]) for g in gev) / steps
            same = bool(torch.equal(dOut, ref))
            macs = float(n) ** 3 / (gemm_ms / 1e3) / 1e12
            out[name] = {"value": ops * steps / (ms / 1e3) / 1e9, "unit": "Gop/s",
                         "ms_per_step": ms / steps, "bit_identical_to_limb": same, "gemm_ms": gemm_ms,
                         "roofline": {"bound": "alu", "achieved": macs, "peak": peaks[kind],
                                      "unit": "T multiply-adds/s", "frac": macs / peaks[kind],
                                      "work": "one multiply-add per (i, j, l) of the product",
                                      "peak_source": f"measured {kind} rate (fm_measure_peak)"}}
        del tA6, tB6, tC6

    # ---- batching form: 4096 independent GEMMs, M, N, K uniform in [32, 512] ----
    if not args.no_batched:
        out["batched"] = run_batched(fm, torch, dev, stream, args)
    # ---- TU decomposition of a rank-10000 16384 x 12288 matrix ----
    if not args.no_tu:
        out["tu"] = run_tu(fm, torch, dev, stream)
    if not args.no_gf2:
        out["gf2"] = run_gf2(fm, torch, dev, stream)
    if not args.no_configs:
        out["configs"] = run_configs(fm, torch, dev, stream, peaks)
        out["curves"] = run_curves(fm, torch, dev, stream)

    # ---- roofline of the dominant kernel (limb GEMM, one launch per step) ----
    burst, sustained, hbm, src = measured_peaks()
    gemm_ms = sorted(kern["limb_gemm"])[len(kern["limb_gemm"]) // 2]
    gemm_avg = sum(kern["limb_gemm"]) / len(kern["limb_gemm"])
    n_products = 3  # Karatsuba on two limbs: A0B0, (A0+A1)(B0+B1), A1B1
    mma_flops = 2.0 * n * n * n * n_products
    achieved = mma_flops / (gemm_avg / 1e3) / 1e12
    traffic = profiled_traffic(os.path.join(ROOT, "paper_1705_04807_gb300", "csrc", "limb_gemm.cu"),
                               "limb_gemm.json", n)
    # the kernel is timed alone between the step's other launches, 2.7 ms a
    # step at full clock: the burst peak is its denominator (the sustained
    # fraction is reported beside it)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": burst, "unit": "TFLOP/s",
                "frac": achieved / burst, "frac_of_sustained": achieved / sustained, "traffic": traffic,
                # three f16 planes of A and of B read once, C read and written
                "algorithmic_bytes": 2.0 * 3 * n * n * 2 + 8.0 * n * n,
                # the library's automatic choice for this shape (fold form,
                # 256-wide tiles): CTA pairs once M, N > 256 and K >= 1024
                "kernel": ("limb_gemm_pair_kernel (cta_group::2, 256 x 256 tiles)" if n > 256 and n >= 1024
                           else "limb_gemm_kernel<256,fold>"),
                "work": f"2*M*N*K*{n_products} f16 MMA flops per launch ({n_products} limb "
                        f"products: Karatsuba on w={w} limbs), n={n}",
                "peak_source": f"bf16 burst, {src} (f16 = bf16 rate); sustained {sustained}",
                "modular_gops": ops / (gemm_avg / 1e3) / 1e9}

    line = {
        "metric": METRIC, "value": value, "unit": "Gop/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32 residues mod p; int8 limbs on f16 tensor cores, f32 exact accumulate",
        "data": "synthetic",
        "config": {"workload": f"C -= (P A Q) * B mod {p}, n={n}, Morton-hybrid T'=128, "
                               "row-major in/out", "n": n, "p": p, "T": 1 << lt_limb,
                   "l2": f"inputs larger than L2 (3 x {4 * n * n >> 20} MiB)"},
        "e2e": e2e_line,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "roofline": roofline,
        "kernels_ms": {k: sum(v) / len(v) for k, v in kern.items()},
    }
    if "batched" in out:
        line["batched"] = out["batched"]
    if "tu" in out:
        # the elimination work against the limb GEMM's modular rate measured in
        # this run (n^3 products at the step's size): the rate a factorization
        # would reach if all of its work ran as that GEMM
        tu = dict(out["tu"])
        tu["roofline"] = {"bound": "limb GEMM rate", "achieved": tu["value"],
                          "peak": roofline["modular_gops"], "unit": "Gop/s",
                          "frac": tu["value"] / roofline["modular_gops"],
                          "peak_source": f"limb GEMM in this run, n={n}, p={p}"}
        line["tu"] = tu
    if "gf2" in out:
        line["gf2"] = out["gf2"]
    if "configs" in out:
        line["configs"] = out["configs"]
        line["curves"] = out["curves"]
    if "plain" in out:
        line["plain"] = out["plain"]
        line["dfma"] = out["dfma"]
        line["limb_over_plain"] = value / out["plain"]["value"]
    # The int8 question: mma.sync s8 carries 8-bit limbs exactly with int32
    # accumulation but needs 4 limb products per modular multiply-add (the
    # Karatsuba digit sums do not fit in 8 bits); the f16 carrier on tcgen05
    # runs at the bf16 burst rate with 3 (Karatsuba).
    if peaks:
        line["peaks"] = dict(peaks, unit="T multiply-adds/s",
                             modular_ceiling_gops={"mma_s8_4_products": 2e3 * peaks["mma_s8"] / 4,
                                                   "tcgen05_f16_3_products": 1e3 * burst / 3})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, secs = cpu_oracle_rate(n, p, target_s=12.0)
        line["cpu_baseline"] = {"value": v, "unit": "Gop/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "seconds": secs}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_case(args):
    """One kernel's call, repeated, for an ncu capture of a small case: the limb
    GEMM (C = A*B mod 65521 or mod 2^31 - 1, n^3), the plain CUDA-core GEMM
    (mod 65521, n^3, T' = --T), the Morton-to-Morton row and column permutation,
    or the permuted row-major -> Morton conversion (n x n)."""
    import numpy as np
    import torch

    import fm_inputs
    import paper_1705_04807_gb300 as fm
    from paper_1705_04807_gb300 import build as fmbuild
    fmbuild.build()
    fm.lib()
    dev = torch.device("cuda", 0)
    if args.case == "tu":  # the TU workload (16384 x 12288, rank 10000; --n = 12288), one factorization
        n = args.n if args.n != N_DEFAULT else 12288
        r = run_tu(fm, torch, dev, torch.cuda.current_stream(), m=(n * 4) // 3, n=n, k=(n * 625) // 768)
        assert r["rank"] == r["rank_expected"], r
        return
    if args.case == "batch":  # the 4096-call workload at T' = --T (--calls fewer), limb plan with planes
        lt = args.T.bit_length() - 1
        big, hi = (16384 if args.calls == 4096 else 8192), 512
        rows, cells = fm_inputs.batch_workload(5, args.calls, 32, hi, big)
        nC = cells * hi
        mats = []
        for q, side in ((1, big), (2, big)):
            x = torch.from_numpy(fm_inputs.uniform_residues(5, (side, side), P, q).view(np.int32)).to(dev)
            t = torch.empty(side * side, dtype=torch.int32, device=dev)
            m = fm.matrix(t, (side >> lt).bit_length() - 1, lt)
            fm.fm_layout_to_morton(x, side, side, side, m)
            mats.append((t, m))
            del x
        tC = torch.zeros(nC * nC, dtype=torch.int32, device=dev)
        mC = fm.matrix(tC, (nC >> lt).bit_length() - 1, lt)
        calls = []
        for c in range(len(rows)):
            M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rows[c])
            call = fm.fm_gemm_call()
            call.C, call.A, call.B = fm.sub(mC, rC, cC, M, N), fm.sub(mats[0][1], rA, cA, M, K), \
                fm.sub(mats[1][1], rB, cB, K, N)
            call.op = fm.FM_OP_SUB
            calls.append(call)
        plan = fm.fm_plan_create(calls, P, fm.FM_ALGO_LIMB_TC)
        for _ in range(args.warmup + args.steps):
            plan.run()
        torch.cuda.synchronize()
        st = fm.fm_get_last_device_status()
        assert st == 0, f"device status {st}"
        plan.close()
        return
    n, lt = args.n, args.T.bit_length() - 1
    lg = (n >> lt).bit_length() - 1
    p = 2147483647 if args.case == "gemm_p31" else P

    def morton(seed, stream):
        x = torch.from_numpy(fm_inputs.uniform_residues(seed, (n, n), p, stream).view(np.int32)).to(dev)
        t = torch.empty(n * n, dtype=torch.int32, device=dev)
        m = fm.matrix(t, lg, lt)
        fm.fm_layout_to_morton(x, n, n, n, m)
        return x, t, m

    if args.case in ("gemm", "gemm_p31", "gemm_plain"):
        mats = [morton(1, q) for q in range(3)]
        subs = [fm.sub(m, 0, 0, n, n) for _, _, m in mats]
        algo = fm.FM_ALGO_PLAIN if args.case == "gemm_plain" else fm.FM_ALGO_LIMB_TC
        call = lambda: fm.fm_gemm_modp(subs[0], subs[1], subs[2], p, fm.FM_OP_SUB, algo)  # noqa: E731
    else:
        x, t0, m0 = morton(1, 0)
        t1 = torch.empty_like(t0)
        m1 = fm.matrix(t1, lg, lt)
        rp = torch.from_numpy(fm_inputs.permutation(1, n, 1)).to(dev)
        cp = torch.from_numpy(fm_inputs.permutation(1, n, 2)).to(dev)
        if args.case == "permute":
            call = lambda: fm.fm_permute_rows_cols(m0, m1, n, n, rp, cp)  # noqa: E731
        else:
            call = lambda: fm.fm_layout_to_morton_permuted(x, n, n, n, rp, cp, m1)  # noqa: E731
    for _ in range(args.warmup + args.steps):
        call()
    torch.cuda.synchronize()
    st = fm.fm_get_last_device_status()
    assert st == 0, f"device status {st}"


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_fm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
