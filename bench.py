"""Benchmark of the tridiagonal -> band eigenvector back-transformation (Eq. 6d).

Default workload: real symmetric, n = 32768, semi-bandwidth 64, nev = 9830
lowest eigenvectors (DFT-like band; the largest single-GPU configuration,
the one the precision form is quoted on). One step = the whole hot path on
one batch: re-lay the reflector store (K = 8,403,968 reflectors) and apply it
to the 32768 x 9830 eigenvector block with the FP64 kernel. Inputs are seeded
and synthetic (unitary Householder reflectors with the exact store geometry,
N(0, 1/n) eigenvector block); both exceed the 129 MB L2.

Metric: algorithmic TFLOP/s = 4 * nev * sum_k L_k flops per step (Eq. 8:
a length-L dot product and a length-L update per reflector and column)
divided by device time. Roofline: the apply kernel is FP64-ALU bound
(arithmetic intensity ~2000 flop/byte, far above the FP64 ridge of ~0.2); its
peak is the FP64 rate measured by the library's probe in the same run, at the
clock sampled while the kernel ran. The same JSON line carries the split-
precision (BF16 tensor-core) form on the same inputs (speed-up over FP64 and
its error against the oracle), and the other configurations as sub-objects:
complex n = 20000, the 64-problem batch against sequential launches, and
n = 512.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank runs an independent replica (the columns
of an eigenvector block are independent; no data-path collective).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2002_10991_gb300 import inputs as I  # noqa: E402

METRIC = "eigvec back-transform TFLOP/s,% FP64 peak; mixed vs FP64 speedup at set resid"
WORKLOAD = "real-n32768-b64-dft"
# the other configurations, measured as sub-objects of the default line
EXTRA_WORKLOADS = ("complex-n20000-b64-dft", "batch-64-mixed", "real-n512-b32-uniform")

# FP64 peak of a GB300: 152 SMs x 2 DFMA per clock x 2 flops at the 2070 MHz
# maximum SM clock (a DFMA microbenchmark measured 1.198 TFLOP/s at ~2000 MHz,
# i.e. the same 2 DFMA/clock/SM).
SMS, DFMA_PER_CLK_SM, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_TFLOPS = SMS * DFMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12

# DRAM bytes (read + write) of one apply-kernel launch on this workload, from
# the ncu capture summarised in profiles/, valid for the kernel sources whose
# hash is recorded beside it (reported as null otherwise).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "apply_kernel_traffic.json")


def bf16_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1900.0  # fallback figure of the profiling recipe


BF16_PEAK_TFLOPS = bf16_peak()


def split_tensor_flops(w):
    """BF16 tensor-core flops the split form issues per step: per WY block of
    32 reflectors and per column, 26 digit-pair products each of (32 x RP) and
    (RP x 32) with RP = b + 31 rounded up to 16 (2 flops per multiply-add)."""
    n, b, nev = w["n"], w["b"], w["nev"]
    nb, pairs = 32, 26
    rp = (b + nb - 1 + 15) // 16 * 16
    J = (n - 2 + b - 1) // b if n >= 3 else 0
    blocks = sum((n - 3 - j * b + 1 + nb - 1) // nb for j in range(J))
    strips = (nev + 63) // 64
    return blocks * strips * 64 * pairs * 2 * (2 * nb * rp)


def tc_tensor_flops(w):
    """BF16 tensor-core flops the tcgen05 split form issues per step: per WY
    block (blocks aligned to stages 32k..32k+31) and per 128-column strip, 26
    digit-pair products in each of the two contractions, each 128 x 32 x RP
    (RP = b + 31 rounded up to 32; 2 flops per multiply-add)."""
    n, b, nev = w["n"], w["b"], w["nev"]
    nb, pairs = 32, 26
    rp = (b + nb - 1 + 31) // 32 * 32
    J = (n - 2 + b - 1) // b if n >= 3 else 0
    blocks = sum((n - 3 - j * b) // nb + 1 for j in range(J))
    strips = (nev + 127) // 128
    return blocks * strips * 2 * pairs * 2 * (128 * nb * rp)


VARIANTS = {"fp64": 0, "split": 1, "split-tc": 2}
# our kernels per timed step: re-layout (+ per-plan preparation), apply (+ the fixed-point conversions)
LAUNCHES_PER_STEP = {"fp64": 2, "split": 5, "split-tc": 5}
SPLIT_KERNEL = {"split": "tbbt::split::split_apply_kernel<{b}>", "split-tc": "tbbt::tcs::tc_apply_kernel<{b}>"}


BATCH_WORKLOAD = "batch-64-mixed"
# band -> tridiagonal on the GPU (the step that produces the store), DFT-like band
BULGE_WORKLOADS = {"bulge-real-n4096-b64": (4096, 64, False), "bulge-complex-n4096-b64": (4096, 64, True),
                   "bulge-real-n8192-b64": (8192, 64, False)}


# band -> full back-transformation (the step after the path): (n, b, nev, complex, seed)
B2F_WORKLOADS = {"b2f-real-n8192-b64-nev4096": (8192, 64, 4096, False, I.SEED_BASE + 8),
                 "b2f-complex-n4096-b64-nev2048": (4096, 64, 2048, True, I.SEED_BASE + 10),
                 "b2f-real-n4096-b64-nev2048": (4096, 64, 2048, False, I.SEED_BASE + 11),
                 # a smaller case of the n=8192 launch configuration (64-row chunks) for profiler captures
                 "b2f-real-n4096-b64-nev4096": (4096, 64, 4096, False, I.SEED_BASE + 12)}


# tridiagonal eigensolver on the GPU (Eq. 6c): the T of a workload's band, nev lowest eigenpairs
TRIDIAG_WORKLOADS = {"tridiag-real-n8192-nev4096": "real-n8192-b64-dft",
                     "tridiag-real-n32768-nev9830": "real-n32768-b64-dft"}


def set_workload(name: str):
    global WORKLOAD
    if name not in I.WORKLOADS and name != BATCH_WORKLOAD and name not in BULGE_WORKLOADS and \
            name not in B2F_WORKLOADS and name not in TRIDIAG_WORKLOADS:
        raise SystemExit(f"unknown workload {name}")
    WORKLOAD = name


def b2f_split_tensor_flops(n: int, b: int, nev: int, sms: int) -> float:
    """BF16 tensor-core flops of the split band -> full form per call: per
    128-column strip, per WY block and per 96-row batch of a slot's 32-row
    tiles, 26 digit-pair products in each contraction (128 x 32 x 96, and
    three of 128 x 32 x 32). Slots and tiles as the library deals them."""
    K1 = max(n - b, 0)
    if K1 == 0 or nev == 0:
        return 0.0
    P_, ntiles, strips = (K1 + 31) // 32, (n + 31) // 32, (nev + 127) // 128
    best, SK = None, 1
    for sk in range(1, min(8, sms) + 1):
        conc = max(sms // sk, 1)
        t = -(-strips // conc) / sk
        if sk == 1 or t < best * 0.999:
            best, SK = t, sk
    batches = 0
    for p in range(P_):
        t0 = (32 * p + b) // 32
        for k in range(SK):
            f = t0 + ((k - t0) % SK)
            cnt = (ntiles - 1 - f) // SK + 1 if f < ntiles else 0
            batches += (cnt + 2) // 3
    per_batch = 26 * 2.0 * 128 * 32 * 96 * 2
    return per_batch * batches * strips


def b2f_bench(args):
    """Band -> full back-transformation (Eq. 6e) on the GPU: one call of the
    C ABI per step (T factors of the 32-reflector blocks, then the apply
    kernel; the split form adds its digit preparation and the fixed-point
    conversions), timed with CUDA events on the calling stream; the oracle on
    the host cores on a column sample; parity on sampled columns."""
    import torch

    import oracle
    import paper_2002_10991_gb300 as P

    torch.cuda.set_device(0)
    n, b, nev, cplx, seed = B2F_WORKLOADS[WORKLOAD]
    if args.variant not in ("fp64", "split-tc") or (cplx and args.variant != "fp64"):
        raise SystemExit("band -> full: --variant fp64, or split-tc for real data")
    variant = VARIANTS[args.variant]
    a, tau = I.synthetic_full_store(n, b, seed, cplx)
    Y = I.eigvec_block(n, nev, seed + 1, cplx)
    da = torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
    dt = torch.from_numpy(tau).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().t()
    cols = np.unique(np.linspace(0, nev - 1, 8).astype(int))
    P.trans_ev_band_to_full(da, dt, n, b, nev, dq, variant=variant)  # parity pass on the original columns
    P.stream_check()
    Cg = dq[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    Co = oracle.back_transform_full(a, tau, n, b, np.asfortranarray(Y[:, cols]), nthreads=oracle.num_cpus())
    err = float(np.abs(Cg - Co).max())
    for _ in range(max(args.warmup, 1)):
        P.trans_ev_band_to_full(da, dt, n, b, nev, dq, variant=variant)
    P.stream_check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            P.trans_ev_band_to_full(da, dt, n, b, nev, dq, variant=variant)
        e1.record(stream)
        torch.cuda.synchronize()
    P.stream_check()
    ms = e0.elapsed_time(e1) / args.steps
    K1 = max(n - b, 0)
    sum_l = K1 * (K1 + 1) // 2  # reflector c has length n - c - b
    flops = (16.0 if cplx else 4.0) * nev * sum_l
    tflops = flops / (ms * 1e-3) / 1e12
    # the oracle on the host cores, on a column sample sized to ~10 s
    cores = oracle.num_cpus()
    ncs = max(cores, 16)
    Ys = np.asfortranarray(Y[:, :ncs])
    t0 = time.perf_counter()
    oracle.back_transform_full(a, tau, n, b, Ys, nthreads=cores)
    cpu_s = time.perf_counter() - t0
    cpu_tf = (16.0 if cplx else 4.0) * ncs * sum_l / cpu_s / 1e12
    if args.variant == "fp64":
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "tbbt::bf::bf_apply_kernel (timed with the T-factor kernel: the whole call)"}
    else:
        tens = b2f_split_tensor_flops(n, b, nev, torch.cuda.get_device_properties(0).multi_processor_count)
        ach = tens / (ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / BF16_PEAK_TFLOPS, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 GEMM burst)",
                "fp64_equivalent_tflops": tflops, "tensor_flops_per_step": tens,
                "kernel": "tbbt::bfs::bfs_apply_kernel (timed with the preparation kernels: the whole call)"}
    line = {
        "metric": "band->full back-transform TFLOP/s (Eq. 6e)", "value": tflops, "unit": "TFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128" if cplx else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nbw": b, "nev": nev, "reflectors": K1,
                   "store": "seeded unitary reflectors, LAPACK layout", "l2": "inputs larger than L2"},
        "roofline": roof,
        "cpu_baseline": {"value": cpu_tf, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"{ncs} of {nev} columns"},
        "parity": {"max_abs_err_vs_oracle": err, "columns": len(cols)},
        "gpu_launches": (2 if args.variant == "fp64" else 7) * args.steps, "clocks": clocks.summary(),
        "variant": args.variant,
    }
    print(json.dumps(line), flush=True)


def tridiag_bench(args):
    """Tridiagonal eigensolver (Eq. 6c) on the GPU for the nev lowest
    eigenpairs of the T that the GPU bulge chase makes of a workload's band:
    time per call; eigenvalues against LAPACK's bisection on the host
    (scipy, timed as the host baseline); residual and orthogonality of the
    vectors on the device."""
    import torch
    from scipy.linalg import eigvalsh_tridiagonal

    import paper_2002_10991_gb300 as P

    torch.cuda.set_device(0)
    src = TRIDIAG_WORKLOADS[WORKLOAD]
    w_ = I.WORKLOADS[src]
    n, b, nev = w_["n"], w_["b"], w_["nev"]
    W = I.band_for(src)
    _, _, d, e = P.bulge_chase(torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t())
    P.stream_check()
    for _ in range(max(args.warmup, 1)):
        w, X = P.tridiag_eig(d, e, nev)
    P.stream_check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            w, X = P.tridiag_eig(d, e, nev)
        e1.record(stream)
        torch.cuda.synchronize()
    P.stream_check()
    ms = e0.elapsed_time(e1) / args.steps
    dh, eh = d.cpu().numpy(), e.cpu().numpy()
    t0 = time.perf_counter()
    lam = eigvalsh_tridiagonal(dh, eh, select="i", select_range=(0, nev - 1))
    host_s = time.perf_counter() - t0
    r = np.abs(dh).copy()
    r[1:] += np.abs(eh)
    r[:-1] += np.abs(eh)
    tn = float(r.max())
    TX = d[:, None] * X
    TX[1:] += e[:, None] * X[:-1]
    TX[:-1] += e[:, None] * X[1:]
    res = torch.linalg.vector_norm(TX - X * w[None, :], dim=0).max().item() / tn
    del TX
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    line = {
        "metric": "tridiagonal eigensolver time (nev lowest eigenpairs)", "value": ms, "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nev": nev, "tridiagonal": f"GPU bulge chase of the {src} band"},
        "parity": {"max_abs_eig_err_vs_lapack_over_tnorm": float(np.abs(w.cpu().numpy() - lam).max() / tn),
                   "residual_max_over_tnorm": res, "orthogonality_max": G.abs().max().item()},
        "host_baseline": {"value": host_s * 1e3, "unit": "ms", "kind": "LAPACK eigenvalues only (scipy stebz)"},
        "gpu_launches": 5 * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def bulge_parity(d, e, do, eo):
    """What is unique in a tridiagonal reduction of this band. The signs of e,
    and with them tau and v, follow the rounding of near-zero bulge entries,
    and d itself moves by ~1e-7 under a 1e-15 relative perturbation of the
    n=8192 band; the spectrum of T and |e| are what two correct reductions
    share."""
    from scipy.linalg import eigvalsh_tridiagonal

    lam = eigvalsh_tridiagonal(d, e) if len(d) > 1 else d
    lam_o = eigvalsh_tridiagonal(do, eo) if len(do) > 1 else do
    return {"max_abs_eig_T": float(np.abs(lam - lam_o).max(initial=0)),
            "max_abs_eig_T_rel": float(np.abs(lam - lam_o).max(initial=0) / max(np.abs(lam_o).max(initial=0), 1e-300)),
            "max_abs_d": float(np.abs(d - do).max(initial=0)),
            "max_abs_abs_e": float(np.abs(np.abs(e) - np.abs(eo)).max(initial=0))}


def bulge_bench(args):
    """Band -> tridiagonal reduction by bulge chasing (Eq. 6b) on the GPU
    against the oracle's reduction on the host (single-threaded C), on a
    seeded DFT-like band; parity of the tridiagonal matrix against the oracle's."""
    import torch

    import paper_2002_10991_gb300 as P

    import oracle

    torch.cuda.set_device(0)
    n, b, cplx = BULGE_WORKLOADS[WORKLOAD]
    W = I.band_dft(n, b, 2002109910 + n, cplx)
    band = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    for _ in range(max(args.warmup, 1)):
        P.bulge_chase(band)
    P.stream_check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            out = P.bulge_chase(band)
        e1.record(stream)
        torch.cuda.synchronize()
    P.stream_check()
    ms = e0.elapsed_time(e1) / args.steps
    d, e = (x.cpu().numpy() for x in out[2:])
    t0 = time.perf_counter()
    _, _, do, eo = oracle.bulge_chase(W)
    cpu_s = time.perf_counter() - t0
    K = int(out[1].numel())
    # real flops of the reduction, counted from the store: a reflector of length L is applied from the
    # right to the L x b block below its diagonal block and from the left to the b columns beside it
    # (4 L b each) and two-sidedly to its L x L diagonal block (4 L^2); a complex flop counts 4
    L = I.store_lengths(n, b, cplx).astype(np.float64)
    flops = float(np.sum((4.0 if cplx else 1.0) * (8 * L * b + 4 * L * L)))
    line = {
        "metric": "band->tridiagonal (bulge chasing) time", "value": ms, "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128" if cplx else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nbw": b, "reflectors": K, "band": "seeded DFT-like band"},
        "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "tbbt::bc::bulge_kernel", "note": "latency-bound: a chain of dependent sweeps"},
        "cpu_baseline": {"value": cpu_s * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": "the whole reduction, single-threaded C"},
        "parity": bulge_parity(d, e, do, eo),
        "speedup_vs_cpu_oracle": cpu_s * 1e3 / ms, "gpu_launches": 3 * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def batch_measure(steps: int, autotune: bool = False):
    """The batched form: 64 problems (N uniform in [1000, 6000], nev = N/2,
    b = 32, even p real, odd p complex) in one persistent graph-replayed
    launch, against the same problems as 64 sequential plan launches. Returns
    a dict of the measurements (inputs built and freed here)."""
    import torch

    import paper_2002_10991_gb300 as P

    specs = I.batch_workload()
    probs, flops = [], 0
    for s in specs:
        n, b, nev, c = s["n"], s["b"], s["nev"], s["complex_"]
        v, tau = I.synthetic_store(n, b, s["seed"], c)
        X = I.eigvec_block(n, nev, s["seed"] + 1, c)
        probs.append((torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda(), n, b, nev,
                      torch.from_numpy(X.T.copy()).cuda().t()))
        flops += (16 if c else 4) * nev * int(I.store_lengths(n, b, c).sum())
    t0 = time.perf_counter()
    batch = P.Batch(probs, autotune=autotune, autotune_cache=os.environ.get("TBBT_AUTOTUNE_CACHE"))
    create_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    batch.execute()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        e0.record(stream)
        for _ in range(steps):
            batch.execute()
        e1.record(stream)
        torch.cuda.synchronize()
    P.stream_check()
    batched_ms = e0.elapsed_time(e1) / steps
    # the same problems, one plain plan launch after another
    plans = [P.Plan(bool(s["complex_"]), s["n"], s["b"], s["nev"]) for s in specs]
    for pl, (dv, dt, n, b, nev, q) in zip(plans, probs):
        pl.set_reflectors(dv, dt)
        pl.execute(q)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for pl, (dv, dt, n, b, nev, q) in zip(plans, probs):
            pl.set_reflectors(dv, dt)
            pl.execute(q)
    e1.record(stream)
    torch.cuda.synchronize()
    P.stream_check()
    seq_ms = e0.elapsed_time(e1) / steps
    info = batch.info()
    batch.close()
    for pl in plans:
        pl.close()
    value = flops / (batched_ms * 1e-3) / 1e12
    return {
        "workload": BATCH_WORKLOAD, "problems": len(specs),
        "n_range": [min(s["n"] for s in specs), max(s["n"] for s in specs)], "nbw": 32, "nev": "n/2",
        "complex_problems": sum(s["complex_"] for s in specs), "flops_per_step": flops, "steps": steps,
        "batched": {"ms": batched_ms, "tflops": value, "launch": info, "create_s": create_s},
        "sequential": {"ms": seq_ms, "tflops": flops / (seq_ms * 1e-3) / 1e12, "launches_per_step": 2 * len(specs)},
        "speedup_vs_sequential": seq_ms / batched_ms, "clocks": clocks.summary(),
    }


def batch_bench(args):
    import torch

    torch.cuda.set_device(0)
    m = batch_measure(args.steps, args.autotune)
    value = m["batched"]["tflops"]
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": m["batched"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+c128", "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "problems", "n_range", "nbw", "nev", "complex_problems",
                                     "flops_per_step")},
        "batched": m["batched"], "sequential": m["sequential"], "speedup_vs_sequential": m["speedup_vs_sequential"],
        "roofline": {"bound": "alu", "achieved": value, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": value / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "tbbt::batch_kernel"},
        "clocks": m["clocks"], "gpu_launches": 1 + 64,
    }
    print(json.dumps(line), flush=True)


def csrc_hash() -> str:
    """Hash of the sources of the FP64 apply kernel and its schedule (the
    recorded DRAM traffic belongs to that kernel only)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2002_10991_gb300", "csrc")
    for f in ("apply_kernels.cuh", "schedule.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes of one apply-kernel launch of ``workload`` from the ncu
    record, or None if there is none for the current kernel sources."""
    try:
        recs = json.load(open(TRAFFIC_FILE))["records"]
    except Exception:
        return None
    h = csrc_hash()
    for rec in recs:
        if rec.get("workload") == workload and rec.get("csrc_hash") == h:
            return rec.get("bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_inputs(name: str):
    w = I.WORKLOADS[name]
    n, b, nev, cplx = w["n"], w["b"], w["nev"], w["complex_"]
    v, tau = I.synthetic_store(n, b, w["seed"], cplx)
    X = I.eigvec_block(n, nev, w["seed"], cplx)
    sum_l = int(I.store_lengths(n, b, cplx).sum())
    flops = (16 if cplx else 4) * nev * sum_l
    return w, v, tau, X, sum_l, flops


def sample_cols(w, sum_l, flops_target: float, lo: int = 16) -> int:
    """Columns of a host sample worth about ``flops_target`` oracle flops
    (a multiple of 16, at least ``lo``, at most nev)."""
    per_col = (16 if w["complex_"] else 4) * max(sum_l, 1)
    c = int(flops_target / per_col) // 16 * 16
    return int(min(max(c, lo), w["nev"]))


def cpu_sample(v, tau, X, w, ncols: int, seed: int = 1):
    """Columns of the workload the oracle back-transforms on the host."""
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(w["nev"], size=min(ncols, w["nev"]), replace=False))
    return cols, np.asfortranarray(X[:, cols])


def run_oracle_sample(v, tau, w, Xs):
    import oracle

    cores = oracle.num_cpus()
    Z = Xs.copy(order="F")
    t0 = time.perf_counter()
    oracle.back_transform(v, tau, w["n"], w["b"], Z, nthreads=cores)
    return Z, time.perf_counter() - t0, cores


def ranks_max(x: float, world: int, device: str = "cuda") -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args, world, rank):
    """The oracle timed on the host cores (rank 0 only), each step a column
    sample of the workload worth about a second of the host's work."""
    if rank != 0:
        return
    w, v, tau, X, sum_l, flops_full = workload_inputs(WORKLOAD)
    ncols = args.ref_cols if args.ref_cols else sample_cols(w, sum_l, 6e10)
    cols, Xs = cpu_sample(v, tau, X, w, ncols)
    fl = (16 if w["complex_"] else 4) * len(cols) * sum_l
    warm = args.warmup if args.warmup_ref is None else args.warmup_ref
    for _ in range(warm):
        run_oracle_sample(v, tau, w, Xs)
    times, cores = [], 1
    for _ in range(args.steps):
        _, dt, cores = run_oracle_sample(v, tau, w, Xs)
        times.append(dt)
    total = sum(times)
    value = fl * len(times) / total / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": warm, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(w), "data": "synthetic",
        "config": config_dict(w, "host cores; oracle sample"),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(cols)} of {w['nev']} columns, all {len(tau)} reflectors, per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def esize(w):
    return 16 if w["complex_"] else 8


def dtype_name(w):
    return "c128" if w["complex_"] else "f64"


def config_dict(w, note="", name=None):
    return {"workload": name or WORKLOAD, "n": w["n"], "nbw": w["b"], "nev": w["nev"],
            "dtype": "complex128" if w["complex_"] else "real64",
            "store": "seeded synthetic unitary reflectors, canonical store layout",
            "x": "seeded N(0,1/n) eigenvector block",
            "l2": f"inputs larger than L2 (q {w['n'] * w['nev'] * esize(w) / 1e6:.0f} MB, store "
                  f"{I.store_lengths(w['n'], w['b'], w['complex_']).size * w['b'] * esize(w) / 1e6:.0f} MB)",
            "parallelism": "replicas", "note": note}


# ---------------------------------------------------------------------------
# the FP64 roofline's denominator, measured in the same run
# ---------------------------------------------------------------------------

def fp64_probe(device: int, kind: int, warps_per_sm: int = 32, seconds: float = 0.4, repeats: int = 3):
    """Rate of the library's FP64 probe (kind 0: FMA chains, kind 1: FP64
    mma.sync m8n8k4) with ``warps_per_sm`` resident warps per SM, with the SM
    clock sampled while it runs."""
    import ctypes

    import torch

    from paper_2002_10991_gb300 import _native

    L = _native.load()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    threads = 256 if warps_per_sm >= 8 else 32 * warps_per_sm
    blocks = sms * max(warps_per_sm * 32 // threads, 1)
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    h = ctypes.c_void_p(int(stream.cuda_stream))
    fl = ctypes.c_double()

    def run(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = L.tbbt_fp64_probe(kind, blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fl), h)
        e1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(f"tbbt_fp64_probe failed with status {st}")
        return e0.elapsed_time(e1), fl.value

    iters = 200
    ms, _ = run(iters)
    iters = max(iters, int(iters * seconds * 1e3 / max(ms, 1e-3)))
    best, flops = None, 0.0
    with ClockSampler(device) as clocks:
        for _ in range(repeats):
            ms, flops = run(iters)
            best = ms if best is None else min(best, ms)
    cs = clocks.summary()
    tf = flops / (best * 1e-3) / 1e12
    return {"kind": ("fma", "mma")[kind], "tflops": tf, "warps_per_sm": warps_per_sm, "ms": best,
            "sm_mhz": cs["sm_mhz"], "reasons": cs["reasons"],
            "flop_per_clk_per_sm": tf * 1e12 / (sms * cs["sm_mhz"] * 1e6) if cs["sm_mhz"] else None}


def fp64_peak(device: int):
    """The FP64 peak of this device: the faster of the two probes (FMA chains
    and FP64 tensor-core products), with the clock it was taken at."""
    runs = [fp64_probe(device, 0), fp64_probe(device, 1)]
    best = max(runs, key=lambda r: r["tflops"])
    return best, runs


def peak_at_clock(probe: dict, sm_mhz):
    """The probe's rate scaled to the clock a kernel ran at (the FP64 rate is
    proportional to the SM clock)."""
    if probe.get("sm_mhz") and sm_mhz:
        return probe["tflops"] * sm_mhz / probe["sm_mhz"]
    return probe["tflops"]


def fp64_peak_bench(args):
    """The probes over a range of resident warps per SM (one JSON line)."""
    import torch

    torch.cuda.set_device(0)
    from paper_2002_10991_gb300 import _native

    _native.load()
    runs = [fp64_probe(0, kind, wps, seconds=0.5) for kind in (0, 1) for wps in (4, 8, 16, 32, 64)]
    best = max(runs, key=lambda r: r["tflops"])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    line = {"metric": "FP64 peak (probe)", "value": best["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": 3, "warmup": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fp64-peak", "sms": sms}, "best": best, "runs": runs,
            "derived_at_max_clock": FP64_PEAK_TFLOPS}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# one FP64 configuration: time, parity on a column sample, rate
# ---------------------------------------------------------------------------

def measure_fp64(name: str, steps: int, warmup: int, parity_cols: int = 8, sweeps_per_block: int = 0,
                 stages_per_step: int = 0):
    """The plain FP64 path on one named workload: re-layout + apply per step,
    CUDA events on the calling stream, parity of a column sample against the
    oracle. Returns a dict (inputs built and freed here)."""
    import torch

    import paper_2002_10991_gb300 as P

    w, v, tau, X, sum_l, flops = workload_inputs(name)
    n, b, nev, cplx = w["n"], w["b"], w["nev"], w["complex_"]
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda()
    q = torch.from_numpy(X.T.copy()).cuda().t()
    plan = P.Plan(cplx, n, b, nev, sweeps_per_block=sweeps_per_block, stages_per_step=stages_per_step)
    cols, Xs = cpu_sample(v, tau, X, w, parity_cols, seed=3)
    plan.set_reflectors(dv, dt)
    plan.execute(q)
    P.stream_check()
    gpu_cols = q[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    for _ in range(warmup):
        plan.set_reflectors(dv, dt)
        plan.execute(q)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(torch.cuda.current_device()) as clocks:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            plan.set_reflectors(dv, dt)
            ev[k][0].record(stream)
            plan.execute(q)
            ev[k][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    P.stream_check()
    ms = t0.elapsed_time(t1) / steps
    apply_ms = sum(a.elapsed_time(z) for a, z in ev) / steps
    info = plan.info()
    plan.close()
    del q, dv, dt
    Zo, cpu_s, cores = run_oracle_sample(v, tau, w, Xs)
    return {"workload": name, "n": n, "nbw": b, "nev": nev, "dtype": dtype_name(w), "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "apply_ms_avg": apply_ms,
            "tflops": flops / (ms * 1e-3) / 1e12, "apply_tflops": flops / (apply_ms * 1e-3) / 1e12,
            "flops_per_step": flops, "launch": info, "clocks": clocks.summary(),
            "parity": {"max_abs_err_vs_oracle": float(np.abs(Zo - gpu_cols).max()), "columns": len(cols)},
            "kernel": "tbbt::apply_kernel<zdouble, -1>" if cplx else
            f"tbbt::apply_kernel<double, {b if b in (32, 64) else 0}>"}


def band_times(W: np.ndarray, Z):
    """B Z for the Hermitian band matrix B in lower band storage W (b+1, n),
    on the device, with Z (n x m) a device tensor: one shifted product per
    diagonal (B is never formed)."""
    import torch

    b = W.shape[0] - 1
    Wd = torch.from_numpy(W).to(Z.device)
    out = Wd[0].real.to(Z.dtype)[:, None] * Z
    for k in range(1, b + 1):
        c = Wd[k, : Z.shape[0] - k][:, None].to(Z.dtype)
        out[k:] += c * Z[:-k]
        out[:-k] += c.conj() * Z[k:]
    return out


def eigen_quality(W: np.ndarray, w, Z, sample: int = 1024, seed: int = 5):
    """Residual max_j ||B z_j - w_j z_j|| / ||B||_2 over all columns, the
    largest deviation of a column norm from 1, and max |z_i^H z_j - delta_ij|
    for a seeded sample of columns against all columns (the whole Z^H Z when
    nev <= sample). ||B||_2 is taken as max_j |w_j| over the computed
    eigenvalues, a lower bound (so the reported residual is an upper bound)."""
    import torch

    nev = Z.shape[1]
    R = band_times(W, Z) - Z * w[None, :]
    bn = max(w.abs().max().item(), np.finfo(float).tiny)
    res = torch.linalg.vector_norm(R, dim=0).max().item() / bn
    del R
    norms = torch.linalg.vector_norm(Z, dim=0)
    if nev <= sample:
        cols = torch.arange(nev, device=Z.device)
    else:
        g = torch.Generator(device="cpu").manual_seed(seed)
        cols = torch.randperm(nev, generator=g)[:sample].sort().values.to(Z.device)
    G = Z[:, cols].conj().t() @ Z
    G[torch.arange(len(cols), device=Z.device), cols] -= 1.0
    return {"residual_max_over_norm": res, "norm": "max |computed eigenvalue| (<= ||B||_2)",
            "max_abs_column_norm_minus_1": (norms - 1.0).abs().max().item(),
            "orthogonality_max": G.abs().max().item(),
            "orthogonality_columns": f"{len(cols)} sampled of {nev} against all" if nev > sample else "all"}


def split_accuracy(name: str):
    """The split-precision form on true eigenvectors at the workload's size:
    GPU bulge chase of the workload's band (Eq. 6b), GPU tridiagonal
    eigensolver (Eq. 6c), then the tcgen05 split-precision back-transform
    (Eq. 6d); residual and orthogonality of the band matrix's eigenpairs."""
    import torch

    import paper_2002_10991_gb300 as P

    w_ = I.WORKLOADS[name]
    n, b, nev = w_["n"], w_["b"], w_["nev"]
    W = I.band_for(name)
    band = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    v, tau, d, e = P.bulge_chase(band)
    ev[1].record(stream)
    w, X = P.tridiag_eig(d, e, nev)
    ev[2].record(stream)
    X64 = X.clone()
    sp = P.Plan(False, n, b, nev, variant=VARIANTS["split-tc"])
    sp.set_reflectors(v, tau)
    sp.execute(X)
    ev[3].record(stream)
    P.stream_check()
    sp.close()
    # the same chain with the FP64 back-transform, for comparison
    P.trans_ev_tridi_to_band(v, tau, n, b, nev, X64)
    P.stream_check()
    P.release_cache()
    del band, v, tau
    q64 = eigen_quality(W, w, X64)
    diff = (X - X64).abs().max().item()
    del X64
    q = eigen_quality(W, w, X)
    q["fp64_back_transform"] = {k: q64[k] for k in ("residual_max_over_norm", "max_abs_column_norm_minus_1",
                                                     "orthogonality_max")}
    q["max_abs_diff_split_vs_fp64"] = diff
    q.update({"chain": "GPU bulge chase -> GPU tridiagonal eigensolver -> split-tc back-transform",
              "workload_band": name, "n": n, "nbw": b, "nev": nev,
              "ms": {"bulge_chase": ev[0].elapsed_time(ev[1]), "tridiag_eig": ev[1].elapsed_time(ev[2]),
                     "split_back_transform": ev[2].elapsed_time(ev[3])}})
    return q


def chain_n512():
    """The plain method on the n = 512 uniform band, all 512 eigenvectors:
    bulge chase, tridiagonal eigensolver and back-transform on the GPU
    against the oracle's bulge chase, implicit QL and back-transform on the
    host (eigenvalues, eigenvectors up to sign, residual, orthogonality)."""
    import torch

    import oracle
    import paper_2002_10991_gb300 as P

    name = "real-n512-b32-uniform"
    w_ = I.WORKLOADS[name]
    n, b, nev = w_["n"], w_["b"], w_["nev"]
    W = I.band_for(name)
    band = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    stream = torch.cuda.current_stream()

    def gpu_chain():
        v, tau, d, e = P.bulge_chase(band)
        w, X = P.tridiag_eig(d, e, nev)
        P.trans_ev_tridi_to_band(v, tau, n, b, nev, X)
        return w, X

    for _ in range(2):
        gpu_chain()
    torch.cuda.synchronize()
    steps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        w, X = gpu_chain()
    e1.record(stream)
    P.stream_check()
    ms = e0.elapsed_time(e1) / steps
    t0 = time.perf_counter()
    v_o, t_o, d_o, e_o = oracle.bulge_chase(W)
    lam_o, Xo = oracle.tridiag_ql(d_o, e_o)
    Zo = oracle.back_transform(v_o, t_o, n, b, np.asfortranarray(Xo[:, :nev]), nthreads=1)
    cpu_ms = (time.perf_counter() - t0) * 1e3
    Zg, wg = X.cpu().numpy(), w.cpu().numpy()
    sgn = np.sign(np.sum(Zg * Zo, axis=0))
    q = eigen_quality(W, w, X)
    q.update({"workload": name, "n": n, "nbw": b, "nev": nev, "steps": steps, "ms_per_chain": ms,
              "chain": "GPU bulge chase -> GPU tridiagonal eigensolver -> GPU back-transform",
              "oracle_chain_ms": cpu_ms, "oracle_chain_cores": 1,
              "max_abs_eigenvalue_err_vs_oracle": float(np.abs(wg - lam_o[:nev]).max()),
              "max_abs_eigvec_err_vs_oracle_up_to_sign": float(np.abs(Zg - Zo * sgn[None, :]).max())})
    return q


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-cols", type=int, default=0,
                    help="columns in the CPU-baseline sample (0: about 5e11 oracle flops' worth)")
    ap.add_argument("--ref-cols", type=int, default=0,
                    help="columns per step of the reference arm (0: about 6e10 oracle flops' worth)")
    ap.add_argument("--warmup-ref", type=int, default=None, help="reference arm warm-ups (default: --warmup)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--split-steps", type=int, default=5,
                    help="fp64 runs of real b=32/64 workloads: also time this many steps of the tcgen05 "
                         "split-precision form on the same inputs (0: skip)")
    ap.add_argument("--extras", default="default",
                    help="comma-separated other configurations measured into the same line "
                         f"({', '.join(EXTRA_WORKLOADS)}); 'default' = all of them for the default workload, "
                         "'none' = skip")
    ap.add_argument("--extra-steps", type=int, default=2, help="timed steps of each extra configuration")
    ap.add_argument("--split-accuracy", type=int, default=1,
                    help="1: residual and orthogonality of the split form on true eigenvectors of the "
                         "workload's band (GPU bulge chase and tridiagonal eigensolver first)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named workload (default: the benchmark workload; others are for profiler captures, "
                         "the batched-form measurement, the FP64 probe sweep (fp64-peak), the GPU bulge chase (" +
                         ", ".join(BULGE_WORKLOADS) + ") and the band -> full back-transformation (" +
                         ", ".join(B2F_WORKLOADS) + "))")
    ap.add_argument("--autotune", action="store_true", help="batched workload: tune the launch geometry first")
    ap.add_argument("--geometry-sweep", default="",
                    help="FP64 workloads: semicolon-separated sweeps_per_block,stages_per_step pairs, each timed "
                         "(--steps steps after one warm-up) into one JSON line instead of the benchmark")
    ap.add_argument("--variant", default="fp64", choices=list(VARIANTS),
                    help="fp64: reflector-by-reflector FP64 kernel; split: WY blocks on BF16 tensor cores "
                         "with exact digit slices (real b=32/64, warp-level mma.sync); split-tc: the same "
                         "on tcgen05 with accumulators in tensor memory; split forms are timed against fp64 "
                         "in the same run")
    args = ap.parse_args()
    default_workload = args.workload == WORKLOAD
    if args.workload == "fp64-peak":
        fp64_peak_bench(args)
        return
    set_workload(args.workload)
    if WORKLOAD == BATCH_WORKLOAD:
        batch_bench(args)
        return
    if WORKLOAD in BULGE_WORKLOADS:
        bulge_bench(args)
        return
    if WORKLOAD in B2F_WORKLOADS:
        b2f_bench(args)
        return
    if WORKLOAD in TRIDIAG_WORKLOADS:
        tridiag_bench(args)
        return
    if args.geometry_sweep:
        import torch

        torch.cuda.set_device(0)
        out = {}
        for pair in args.geometry_sweep.split(";"):
            G, NB = (int(x) for x in pair.split(","))
            m = measure_fp64(WORKLOAD, args.steps, 1, parity_cols=8, sweeps_per_block=G, stages_per_step=NB)
            out[pair] = {"ms": m["apply_ms_avg"], "tflops": m["apply_tflops"], "launch": m["launch"],
                         "parity": m["parity"]["max_abs_err_vs_oracle"], "clocks": m["clocks"]}
        print(json.dumps({"metric": "launch geometry sweep", "config": {"workload": WORKLOAD}, "runs": out}),
              flush=True)
        return
    world, rank, local = dist_setup()

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
        reference_arm(args, world, rank)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    import torch

    import paper_2002_10991_gb300 as P
    from paper_2002_10991_gb300 import _native

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _native.load()  # the library must be built (fails loudly otherwise)

    probe, probe_runs = fp64_peak(local)

    w, v, tau, X, sum_l, flops = workload_inputs(WORKLOAD)
    n, b, nev, cplx = w["n"], w["b"], w["nev"], w["complex_"]
    es = esize(w)
    dv = torch.from_numpy(v).cuda()
    dt = torch.from_numpy(tau).cuda()
    q = torch.from_numpy(X.T.copy()).cuda().t()
    stream = torch.cuda.current_stream()
    split = args.variant != "fp64"
    plan = P.Plan(cplx, n, b, nev, variant=VARIANTS[args.variant])
    info = plan.info()

    # parity pass on the pristine block (columns checked by the CPU baseline)
    ncpu = args.cpu_cols if args.cpu_cols else sample_cols(w, sum_l, 5e11)
    cols, Xs = cpu_sample(v, tau, X, w, ncpu)
    plan.set_reflectors(dv, dt)
    plan.execute(q)
    P.stream_check()
    gpu_cols = q[:, torch.from_numpy(cols).cuda()].cpu().numpy()

    for _ in range(args.warmup):
        plan.set_reflectors(dv, dt)
        plan.execute(q)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for k in range(args.steps):
            a, m, z = ev[k]
            a.record(stream)
            plan.set_reflectors(dv, dt)
            m.record(stream)
            plan.execute(q)
            z.record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    P.stream_check()
    total_ms = t_begin.elapsed_time(t_end)
    apply_ms = [m.elapsed_time(z) for (a, m, z) in ev]
    relayout_ms = [a.elapsed_time(m) for (a, m, z) in ev]
    total_ms = ranks_max(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = flops * args.steps * world / (total_ms * 1e-3) / 1e12

    # the mixed-precision form on the same inputs (headline: speedup over FP64 at the set accuracy)
    split_tc = None
    if not split and not cplx and b in (32, 64) and args.split_steps > 0:
        sp = P.Plan(cplx, n, b, nev, variant=VARIANTS["split-tc"])
        qs = torch.from_numpy(X.T.copy()).cuda().t()
        sp.set_reflectors(dv, dt)
        sp.execute(qs)
        P.stream_check()
        split_cols = qs[:, torch.from_numpy(cols).cuda()].cpu().numpy()
        for _ in range(2):
            sp.set_reflectors(dv, dt)
            sp.execute(qs)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as sclocks:
            s0.record(stream)
            for _ in range(args.split_steps):
                sp.set_reflectors(dv, dt)
                sp.execute(qs)
            s1.record(stream)
            torch.cuda.synchronize()
        P.stream_check()
        split_tc = {"ms_per_step": s0.elapsed_time(s1) / args.split_steps, "steps": args.split_steps,
                    "cols": split_cols, "clocks": sclocks.summary()}
        sp.close()
        del qs
        if args.split_accuracy and w["kind"] == "dft":
            torch.cuda.empty_cache()
            split_tc["accuracy"] = split_accuracy(WORKLOAD)
            torch.cuda.empty_cache()

    fp64_cmp = None
    if split:
        ref = P.Plan(cplx, n, b, nev)
        ref.set_reflectors(dv, dt)
        qr = q.clone()
        ref.execute(qr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ref.set_reflectors(dv, dt)
        ref.execute(qr)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1)
        fp64_cmp = {"fp64_ms_per_step": fp64_ms, "speedup_vs_fp64": fp64_ms / ms_per_step}
        ref.close()
        del qr

    # end to end through the host-buffer C ABI (pinned host memory, copies inside)
    hv = torch.from_numpy(v).pin_memory()
    ht = torch.from_numpy(tau).pin_memory()
    hq = torch.from_numpy(X.T.copy()).pin_memory().t()
    if split:
        # the plan API with host-side copies around it (the one-shot host call runs the FP64 kernel)
        def e2e_step():
            dv.copy_(hv, non_blocking=True)
            dt.copy_(ht, non_blocking=True)
            q.copy_(hq, non_blocking=True)
            plan.set_reflectors(dv, dt)
            plan.execute(q)
            hq.copy_(q, non_blocking=True)
        api = f"tbbt_plan_set_reflectors + tbbt_plan_execute ({args.variant} variant), pinned host copies"
    else:
        def e2e_step():
            P.trans_ev_tridi_to_band_host(hv, ht, n, b, nev, hq, synchronize=False)
        api = "tbbt_trans_ev_tridi_to_band_host_z" if cplx else "tbbt_trans_ev_tridi_to_band_host_d"
    e2e_step()  # warm (allocates the cached copies)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    P.stream_check()
    e2e_s = time.perf_counter() - t0
    e2e_s = ranks_max(e2e_s, world)
    e2e = {"value": flops * args.e2e_steps * world / e2e_s / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(v.nbytes + tau.nbytes + n * nev * es), "d2h_bytes_per_step": int(n * nev * es),
           "steps": args.e2e_steps, "api": api}
    P.release_cache()
    plan.close()
    del hv, ht, hq, q, dv, dt

    # the other configurations, each as a sub-object of the same line
    extras = {}
    names = []
    if args.extras == "default":
        names = list(EXTRA_WORKLOADS) if default_workload and not split else []
    elif args.extras != "none":
        names = [x for x in args.extras.split(",") if x]
    if rank == 0:
        for nm in names:
            torch.cuda.empty_cache()
            if nm == BATCH_WORKLOAD:
                m = batch_measure(args.extra_steps, autotune=True)
                m["of_fp64_peak"] = m["batched"]["tflops"] / peak_at_clock(probe, m["clocks"]["sm_mhz"])
            elif nm == "real-n512-b32-uniform":
                m = measure_fp64(nm, max(args.extra_steps, 5), 2, parity_cols=512)
                m["of_fp64_peak"] = m["apply_tflops"] / peak_at_clock(probe, m["clocks"]["sm_mhz"])
                m["gpu_chain"] = chain_n512()
            else:
                m = measure_fp64(nm, args.extra_steps, 0, parity_cols=8)
                m["of_fp64_peak"] = m["apply_tflops"] / peak_at_clock(probe, m["clocks"]["sm_mhz"])
            extras[nm] = m

    if rank == 0:
        apply_avg = sum(apply_ms) / len(apply_ms)
        achieved = flops / (apply_avg * 1e-3) / 1e12
        cs = clocks.summary()
        peak = peak_at_clock(probe, cs["sm_mhz"])
        derived_at_clock = SMS * DFMA_PER_CLK_SM * 2 * cs["sm_mhz"] * 1e6 / 1e12 if cs["sm_mhz"] else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None if split else recorded_traffic(WORKLOAD),
                "kernel": "tbbt::apply_kernel<zdouble, -1>" if cplx else f"tbbt::apply_kernel<double, {b if b in (32, 64) else 0}>",
                "peak_source": f"measured: library FP64 probe ({probe['kind']}, {probe['tflops']:.4f} TFLOP/s at "
                               f"{probe['sm_mhz']} MHz) scaled to the {cs['sm_mhz']} MHz sampled during the timed steps",
                "fp64_probe": probe_runs,
                "peak_derived": derived_at_clock,
                "frac_of_derived": achieved / derived_at_clock if derived_at_clock else None,
                "peak_derived_source": "152 SMs x 2 DFMA/clk x 2 flop x sampled SM clock",
                "algorithmic_bytes_per_launch": int(2 * n * nev * es + sum_l * es)}
        Zo, cpu_s, cores = run_oracle_sample(v, tau, w, Xs)
        cpu = {"value": (16 if cplx else 4) * len(cols) * sum_l / cpu_s / 1e12, "unit": "TFLOP/s", "cores": cores,
               "kind": "oracle",
               "sample": f"{len(cols)} of {nev} columns, all {len(tau)} reflectors",
               "parity_max_abs_vs_gpu": float(np.abs(Zo - gpu_cols).max())}
        # the same oracle on one host thread, on the first 16 columns of the sample
        import oracle

        Z1 = np.asfortranarray(Xs[:, :16])
        t0 = time.perf_counter()
        oracle.back_transform(v, tau, n, b, Z1, nthreads=1)
        t1 = time.perf_counter() - t0
        cpu["single_thread"] = {"value": (16 if cplx else 4) * Z1.shape[1] * sum_l / t1 / 1e12, "unit": "TFLOP/s",
                                "cores": 1, "sample": f"{Z1.shape[1]} of {nev} columns, all {len(tau)} reflectors"}
        if split:
            # the BF16 tensor-core form: FP64-equivalent algorithmic rate; its own roofline is the
            # tensor pipe (bf16 MMA issued per step), reported beside the FP64 reference
            tensor_flops = tc_tensor_flops(w) if args.variant == "split-tc" else split_tensor_flops(w)
            roof.update({"bound": "tensor", "kernel": SPLIT_KERNEL[args.variant].format(b=b),
                         "achieved": tensor_flops / (apply_avg * 1e-3) / 1e12, "peak": BF16_PEAK_TFLOPS,
                         "frac": tensor_flops / (apply_avg * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 GEMM burst)",
                         "fp64_equivalent_tflops": achieved, "tensor_flops_per_step": tensor_flops})
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name(w), "data": "synthetic", "config": config_dict(w),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": LAUNCHES_PER_STEP[args.variant] * args.steps,
            "clocks": cs, "relayout_ms_avg": sum(relayout_ms) / len(relayout_ms), "apply_ms_avg": apply_avg,
            "of_fp64_peak": value / peak if not split else None,
            "launch": info, "variant": {"fp64": "fp64", "split": "split_bf16", "split-tc": "split_bf16_tc"}[args.variant],
        }
        if fp64_cmp:
            line.update(fp64_cmp)
        if split_tc:
            sms = split_tc["ms_per_step"]
            line["split_tc"] = {
                "variant": "split_bf16_tc", "kernel": f"tbbt::tcs::tc_apply_kernel<{b}>",
                "ms_per_step": sms, "steps": split_tc["steps"], "speedup_vs_fp64": ms_per_step / sms,
                "fp64_equivalent_tflops": flops / (sms * 1e-3) / 1e12,
                "tensor_tflops": tc_tensor_flops(w) / (sms * 1e-3) / 1e12,
                "tensor_frac_of_bf16_peak": tc_tensor_flops(w) / (sms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                "max_abs_err_vs_oracle": float(np.abs(Zo - split_tc["cols"]).max()),
                "err_sample": cpu["sample"], "clocks": split_tc["clocks"],
            }
            if "accuracy" in split_tc:
                line["split_tc"]["accuracy_true_eigenvectors"] = split_tc["accuracy"]
        if extras:
            line["configs"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
