#!/usr/bin/env python3
"""Benchmark: top-k diffusion-map eigenpairs per second on GB300.

Workload (the paper's s-curve experiment scaled to its largest size, Section 4):
100,000 s-curve points in R^3 (seeded synthetic data), Gaussian kernel with
eps = median squared pairwise distance, alpha = 1, H-matrix with leaf 512,
max rank 128, tol 1e-5, top-20 eigenpairs by Lanczos (nrhs = 1).

One step = the whole path through the C ABI: dm_create (bandwidth, degrees),
dm_compress (tree, skeletons, packing), dm_eigs (Lanczos with the H-matvec,
Ritz vectors), dm_destroy. `value` is eigenpairs/s with the points already in
HBM; `e2e` is the same through host buffers (points from pinned host memory,
eigenvalues and eigenvectors back to the host inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank solves its own cloud
(replicas: the solve has no data-path exchange) and value sums over ranks.

`cpu_baseline` times the FP64 oracle's whole pipeline on the same workload on the
host cores; `--impl reference` times that pipeline once per step, on fewer points
(phase times scaled to N) when the steps would not fit in about two minutes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "s-curve N=100000 d=3, eps=median sq. distance, alpha=1, leaf 512, rank 128, tol 1e-5, "
                        "top-20, nrhs=1", "N": 100_000, "d": 3, "leaf": 512, "rank": 128, "tol": 1e-5, "k": 20}
METRIC = "top-k diffusion-map eigenpairs/s (N=100k s-curve, k=20)"
UNIT = "eigenpairs/s"
# the oracle's full pipeline at the workload's N takes roughly 10 s on 16 host cores (the
# O(N^2) degree passes dominate); the reference arm sizes its per-step samples so that all
# of its steps fit in about two minutes
ORACLE_FULL_S = 10.0
REFERENCE_BUDGET_S = 330.0


def reference_sample_n(steps: int, full_s: float = ORACLE_FULL_S) -> int:
    """Points per timed oracle step of the reference arm: the full workload when the timed
    steps fit the budget at full size (full_s: the predicted seconds of one full-size step;
    30 steps of about 9 s fit on the GPU machine's 16 host cores), else fewer (time grows as n^2
    through the degree passes)."""
    per_step = REFERENCE_BUDGET_S / max(1, steps)
    n = int(WORKLOAD["N"] * min(1.0, math.sqrt(per_step / max(full_s, 1e-3))))
    return max(10_000, n // 1000 * 1000)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=WORKLOAD["N"], help="override N (testing only)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-block", action="store_true", help="skip the block H-matvec and scaling-workload lines")
    p.add_argument("--sections", default="accuracy,precision,block_matvec,block_lanczos,scaling_workload,"
                                         "mnist_workload,batched_clouds",
                   help="comma list of the side measurements to run after the headline")
    p.add_argument("--skip-headline", action="store_true",
                   help="profiling only: run just the side measurements (no timed headline steps)")
    p.add_argument("--serve-requests", type=int, default=2000,
                   help="requests in the timed serving run (after warm-up); 0 skips it")
    p.add_argument("--serve-rate", type=float, default=200.0, help="mean Poisson arrival rate, requests/s")
    p.add_argument("--serve-slots", type=int, default=8)
    p.add_argument("--serve-dims", default="3,64,784", help="point dimensions in the request mix")
    return p.parse_args()


# ------------------------------------------------------------------ clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ serving: Poisson arrivals of mixed requests

SERVE_MIX = ("N log-uniform in [2000, 100000], d from {dims} (s-curve for d=3, 8-component Gaussian mixture "
             "for d=64, MNIST-shaped for d=784), k uniform in [5, 32], tol from {{1e-4, 1e-5}}, leaf 512, rank 128, "
             "eigenvectors returned")


def serve_run(dm, n_req: int, rate: float, slots: int, dims: list[int], warm: int = 100, seed: int = 7,
              max_arrival_s: float = 40.0, max_drain_s: float = 30.0) -> dict:
    """Submit warm + n_req requests at Poisson arrival times through dm_submit and collect them with
    dm_poll; latency = submit to done on the library's clock. Each request's points are a random
    window of a seeded 200,000-point cloud of its dimension (generated once, before timing).
    Bounded: arrivals stop after max_arrival_s and the queue is drained for at most
    max_drain_s (then cancelled). A run is reported as saturated when requests were cancelled
    or never submitted, or when requests completed at less than 95% of the arrival rate (the
    queue then grows and latency measures backlog, not service)."""
    import numpy as np

    import synth

    g = np.random.default_rng(seed)
    base = {}
    for d in dims:
        if d == 3:
            base[d] = synth.as_f32(synth.s_curve(200_000, seed=11))
        elif d == 784:
            base[d] = synth.as_f32(synth.mnist_like(200_000, seed=11))
        else:
            base[d] = synth.as_f32(synth.gaussian_mixture(200_000, d=d, seed=11))
    total = warm + n_req
    Ns = np.exp(g.uniform(np.log(2000), np.log(100_000), size=total)).astype(np.int64)
    ds = g.choice(dims, size=total)
    ks = g.integers(5, 33, size=total)
    tols = g.choice([1e-4, 1e-5], size=total)
    offs = [int(g.integers(0, 200_000 - n + 1)) for n in Ns]
    gaps = g.exponential(1.0 / rate, size=total)
    dm.dm_serve_start(slots=slots, hbm_budget_bytes=150_000_000_000)
    pending, done = {}, {}

    def collect():
        for t in list(pending):
            fin, r = dm.dm_poll(t)
            if fin:
                done[t] = (pending.pop(t), r["status"], r["k"], r["submit_ms"], r["start_ms"], r["done_ms"],
                           r["built_ms"])
                dm.dm_release(t)

    submitted = 0
    try:
        t0 = time.perf_counter()
        due = 0.0
        for i in range(total):
            due += gaps[i]
            if due > max_arrival_s:
                break
            while time.perf_counter() - t0 < due:
                collect()
                time.sleep(0.0002)
            n, d = int(Ns[i]), int(ds[i])
            t = dm.dm_submit(base[d][offs[i]:offs[i] + n], eps=-1.0, alpha=1.0, tol=float(tols[i]), leaf_size=512,
                             max_rank=128, k=int(ks[i]), want_vectors=True, seed=i)
            pending[t] = i
            submitted += 1
        t1 = time.perf_counter()
        while pending and time.perf_counter() - t1 < max_drain_s:
            collect()
            time.sleep(0.0005)
    finally:
        dm.dm_serve_stop()
    cancelled = len(pending)
    rec = sorted(done.values())[warm:]
    lat = np.array([r[5] - r[3] for r in rec])
    ok = [r for r in rec if r[1] == 0]
    span_s = (max(r[5] for r in rec) - min(r[3] for r in rec)) / 1e3
    by_d = {}
    for r in rec:
        by_d.setdefault(int(ds[r[0]]), []).append(r[5] - r[3])
    return {"requests": len(rec), "warmup_requests": warm, "submitted": submitted, "cancelled_at_stop": cancelled,
            "saturated": bool(cancelled or submitted < total or len(rec) / span_s < 0.95 * rate),
            "completion_over_arrival_rate": (len(rec) / span_s) / rate, "rate_per_s": rate, "slots": slots,
            "mix": SERVE_MIX.format(dims=sorted(set(int(x) for x in dims))),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_components_ms": {"queue": float(np.percentile([r[4] - r[3] for r in rec], 50)),
                                  "build": float(np.percentile([r[6] - r[4] for r in rec], 50)),
                                  "eigensolve": float(np.percentile([r[5] - r[6] for r in rec], 50))},
            "mean_ms": float(lat.mean()), "eigenpairs_per_s": float(sum(r[2] for r in ok) / span_s),
            "requests_per_s": len(rec) / span_s, "not_converged": sum(r[1] == -4 for r in rec),
            "failed": sum(r[1] not in (0, -4) for r in rec),
            "p50_ms_by_d": {str(d): float(np.percentile(v, 50)) for d, v in sorted(by_d.items())},
            "p99_ms_by_d": {str(d): float(np.percentile(v, 99)) for d, v in sorted(by_d.items())},
            "hbm_budget_gb": 150}


# ------------------------------------------------------------------ accuracy against FP64

_FP64_REF = {}


def fp64_reference(X, W) -> dict:
    """FP64 reference eigenpairs of the workload from the oracle on the host cores: the exact
    degrees, an H-matrix at tol 1e-9 (eigenvalue error ~3e-8 relative against the dense
    solve at 10,000 points) and Lanczos to residual 1e-11. Computed once per process."""
    if "ev" in _FP64_REF:
        return _FP64_REF
    import oracle as O

    O.build()
    t0 = time.perf_counter()
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, W["leaf"], 1e-9, W["rank"])
    ev, V, it, st = O.lanczos_hmat(X, eps, s, H, W["k"], conv_tol=1e-11)
    _FP64_REF.update(ev=ev, V=V, dg=dg, s=s, eps=eps, converged=st == 0, seconds=time.perf_counter() - t0,
                     what="FP64 oracle: exact degrees, H-matrix at tol 1e-9 (leaf %d, rank %d), Lanczos to "
                          "residual 1e-11, on the host cores" % (W["leaf"], W["rank"]))
    return _FP64_REF


def _subspace_angle(A, B) -> float:
    import numpy as np

    sv = np.linalg.svd(A.T @ B, compute_uv=False)
    return math.acos(min(1.0, float(sv.min())))


def accuracy_errors(ref: dict, ev, V, psi=None, t: int = 1) -> dict:
    """Errors of one solve against the FP64 reference: max relative eigenvalue error, the
    largest principal angle between the top-k subspaces, and (psi given) the largest relative
    column error of the diffusion coordinates theta^t Dg^-1/2 phi."""
    import numpy as np

    import oracle as O

    ev = np.asarray(ev, np.float64)
    V = np.asarray(V, np.float64)
    out = {"max_rel_eigenvalue_error": float(np.max(np.abs(ev - ref["ev"]) / np.abs(ref["ev"]))),
           "subspace_angle_rad": _subspace_angle(V, ref["V"])}
    if psi is not None:
        want = O.diffusion_coords(ref["ev"], ref["V"], ref["dg"], t)
        psi = np.asarray(psi, np.float64)
        errs = []
        for i in range(want.shape[1]):
            sgn = 1.0 if np.dot(psi[:, i], want[:, i]) >= 0 else -1.0
            errs.append(np.linalg.norm(sgn * psi[:, i] - want[:, i]) / np.linalg.norm(want[:, i]))
        out["max_rel_coords_error_t1"] = float(max(errs))
    return out


def accuracy_run(dm, torch, stream, X, W, steps: int = 5, tols=None, blocks=(0, 4)) -> dict:
    """The accuracy target against FP64, per compression tolerance and eigensolver: the
    single-vector FP32 Lanczos (block 0) and block Lanczos with 4 vectors per step (FP32
    H-matvec of 4 right-hand sides, FP64 Gram-Schmidt and Cholesky coefficients, FP64
    Rayleigh-Ritz), each with its eigenvalue, subspace-angle and diffusion-coordinate errors
    against the FP64 reference and its throughput (create + compress + eigs + destroy, points
    in HBM, CUDA events), at the workload's tolerance (1e-5) and at 3e-7 (the loosest
    tolerance whose eigenvalues stay within 1e-5 relative of FP64 on this workload)."""
    import numpy as np

    Xd = torch.from_numpy(X).cuda()
    res = {}
    tols = tols or (W["tol"], 3e-7)
    for tol in tols:
        for b in blocks:
            cfg = dm.dm_config_default(stream=stream.cuda_stream, block_size=b)
            ts, te = [], []
            for i in range(steps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h = dm.dm_create(Xd, eps=-1.0, alpha=1.0, cfg=cfg)
                dm.dm_compress(h, tol, W["leaf"], W["rank"])
                ev, V, conv = dm.dm_eigs(h, W["k"], evecs=True, device_out=True)
                st = dm.dm_get_stats(h)
                if i == steps + 1:
                    psi = dm.dm_coords(h, W["k"], 1)
                    Vh = V.cpu().numpy()
                dm.dm_destroy(h)
                e1.record(stream)
                e1.synchronize()
                if i >= 2:
                    ts.append(e0.elapsed_time(e1))
                    te.append(st["ms_eigs"])
            ms = statistics.median(ts)
            res[f"tol_{tol:g}_block{b}"] = {
                "solver": "single-vector Lanczos, FP32 H-matvec" if b == 0 else
                          f"block Lanczos, {b} vectors per step: FP32 H-matvec of {b} right-hand sides, FP64 "
                          "Gram-Schmidt/Cholesky coefficients and Rayleigh-Ritz",
                "ms_per_solve": ms, "eigenpairs_per_s": W["k"] / (ms * 1e-3), "ms_eigs": statistics.median(te),
                "converged": bool(conv), "basis_vectors": st["lanczos_iters"],
                "ranks": {"min": st["rank_min"], "max": st["rank_max"], "mean": round(st["rank_mean"], 2)},
                "phases_ms": {key: round(float(st[key]), 3) for key in
                              ("ms_create", "ms_degrees", "ms_tree", "ms_skeleton", "ms_pack", "ms_eigs")},
                "hmatvec_path": st["hmatvec_path"],
                "_ev": np.asarray(ev), "_V": Vh, "_psi": psi}
    ref = fp64_reference(X, W)
    for key, r in res.items():
        r.update(accuracy_errors(ref, r.pop("_ev"), r.pop("_V"), r.pop("_psi")))
        r["meets_1e-5_rel_and_1e-3_rad"] = bool(r["max_rel_eigenvalue_error"] <= 1e-5
                                               and r["subspace_angle_rad"] <= 1e-3)
    for tol in tols:
        base = res.get(f"tol_{tol:g}_block0")
        for b in blocks:
            r = res.get(f"tol_{tol:g}_block{b}")
            if b and base and r:
                r["eigs_speedup_vs_single_vector"] = base["ms_eigs"] / r["ms_eigs"]
                r["solve_speedup_vs_single_vector"] = base["ms_per_solve"] / r["ms_per_solve"]
    res["reference"] = ref["what"]
    res["reference_s"] = round(ref["seconds"], 1)
    res["note"] = ("errors against FP64 combine the approximation of S by the H-matrix (set by tol: Eq. 1.1 "
                   "bounds it relative to |S| = 1, so the smallest wanted eigenvalue, ~2.4e-3, carries about "
                   "tol x 20 relative error) and the FP32 arithmetic of the path")
    return res


# ------------------------------------------------------------------ block H-matvec (nrhs > 1)

def _time_matvec(dm, torch, stream, h, x, reps: int) -> float:
    """Median device time (ms) of dm_matvec(h, x) on device-resident x, CUDA events on the
    handle's stream (the near field's side stream joins it before the call returns)."""
    y = torch.empty_like(x)
    for _ in range(2):
        dm.dm_matvec(h, x, y)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dm.dm_matvec(h, x, y)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def block_run(dm, torch, stream, X, W) -> dict:
    """The block H-matvec at the bench workload against the single-vector path: nrhs = 16
    (FP32, the block-Lanczos width) and nrhs = 256 (TF32 tensor cores), per right-hand side."""
    out = {}
    N = X.shape[0]
    g = torch.Generator(device="cuda").manual_seed(3)
    for prec, name in ((dm.DM_PREC_FP32, "fp32"), (dm.DM_PREC_TF32, "tf32")):
        cfg = dm.dm_config_default(stream=stream.cuda_stream, block_precision=prec, near_mode=dm.DM_NEAR_CACHED)
        h = dm.dm_create(X, eps=-1.0, alpha=1.0, cfg=cfg)
        dm.dm_compress(h, W["tol"], W["leaf"], W["rank"])
        if name == "fp32":
            x1 = torch.rand(N, device="cuda", generator=g) * 2 - 1
            out["single_vector_ms"] = _time_matvec(dm, torch, stream, h, x1, 20)
        for nrhs in ((16, 64) if name == "fp32" else (16, 64, 256)):
            xb = (torch.rand(nrhs, N, device="cuda", generator=g) * 2 - 1).t()
            ms = _time_matvec(dm, torch, stream, h, xb, 10)
            out[f"{name}_nrhs{nrhs}_ms"] = ms
            out[f"{name}_nrhs{nrhs}_speedup_vs_single_vector"] = out["single_vector_ms"] * nrhs / ms
        dm.dm_destroy(h)
    out["note"] = ("dm_matvec on device-resident blocks, CUDA-event median; speedup = nrhs single-vector "
                   "H-matvecs (the nrhs=1 path) over one block call of the same nrhs")
    return out


def block_lanczos_run(dm, stream, X, W, reps: int = 3) -> dict:
    """dm_eigs (top-k) by block Lanczos against the single-vector FP32 Lanczos on the same
    compressed operator: device time of the eigensolve phase (median over reps) and the
    largest relative eigenvalue difference between the two. Block 4 runs the narrow-block
    path (three chained launches per H-matvec, one cooperative launch per step); blocks 8
    and 16 the general block path (per-level tree launches), FP32 or TF32 tensor-core near
    field."""
    res = {}
    ref = None
    for b, prec, name in ((0, dm.DM_PREC_FP32, "single_vector_fp32"), (4, dm.DM_PREC_FP32, "block4_fp32"),
                          (8, dm.DM_PREC_FP32, "block8_fp32"), (16, dm.DM_PREC_FP32, "block16_fp32"),
                          (16, dm.DM_PREC_TF32, "block16_tf32")):
        cfg = dm.dm_config_default(stream=stream.cuda_stream, block_size=b, block_precision=prec,
                                   near_mode=dm.DM_NEAR_CACHED)
        h = dm.dm_create(X, eps=-1.0, alpha=1.0, cfg=cfg)
        dm.dm_compress(h, W["tol"], W["leaf"], W["rank"])
        ts = []
        for _ in range(reps):
            ev, _, conv = dm.dm_eigs(h, W["k"], evecs=True, device_out=True)
            st = dm.dm_get_stats(h)
            ts.append(st["ms_eigs"])
        r = {"ms_eigs": statistics.median(ts), "basis_vectors": st["lanczos_iters"], "converged": bool(conv)}
        if ref is None:
            ref = ev
        else:
            r["max_rel_eig_diff_vs_single_vector"] = float(max(abs(a - c) / abs(c) for a, c in zip(ev, ref)))
            r["speedup_vs_single_vector"] = res["single_vector_fp32"]["ms_eigs"] / r["ms_eigs"]
        res[name] = r
        dm.dm_destroy(h)
    return res


def precision_run(dm, torch, stream, X, W, reps: int = 10) -> dict:
    """The precision matrix of the near field on the bench workload: FP32 (CUDA cores), TF32 and
    split TF32 (three products of TF32 high and low parts; tcgen05, FP32 accumulation). For each:
    the block H-matvec at nrhs 16 and 64 (device time, and the error against the FP64 oracle's
    evaluation of the same compressed structure, max |y - y_fp64| / max |x|), and block Lanczos
    with 16 vectors (eigensolve time, eigenvalue and subspace-angle errors against the FP64
    reference solve)."""
    import numpy as np

    import oracle as O

    O.build()
    ref = fp64_reference(X, W)
    eps = ref["eps"]
    s_host = _FP64_REF.get("s")
    if s_host is None:
        _, _, s_host = O.degrees(X, eps, 1.0)
        _FP64_REF["s"] = s_host
    Hs = O.compress(X, eps, s_host, W["leaf"], W["tol"], W["rank"])
    N = X.shape[0]
    g = np.random.default_rng(7)
    xs = {nb: np.asfortranarray((g.random((N, nb)) * 2 - 1).astype(np.float32)) for nb in (16, 64)}
    yref = {nb: O.hmatvec(X, eps, s_host, Hs, xs[nb][:, :16].astype(np.float64)) for nb in (16,)}
    out = {"structure": "the oracle's FP64 compression (tol %g, leaf %d, rank %d), loaded with dm_load_hmatrix"
                        % (W["tol"], W["leaf"], W["rank"])}
    for prec, name in ((dm.DM_PREC_FP32, "fp32"), (dm.DM_PREC_TF32, "tf32"), (dm.DM_PREC_TF32X3, "tf32x3")):
        r = {}
        cfg = dm.dm_config_default(stream=stream.cuda_stream, block_precision=prec, near_mode=dm.DM_NEAR_CACHED)
        h = dm.dm_create(X, eps=eps, alpha=1.0, cfg=cfg)
        dm.dm_load_hmatrix(h, Hs.L, Hs.max_rank, Hs.perm, Hs.ranks, Hs.skel, Hs.P.astype(np.float32))
        for nb in (16, 64):
            xd = torch.from_numpy(xs[nb]).cuda()
            xd = xd.t().contiguous().t() if nb > 1 else xd
            r[f"nrhs{nb}_ms"] = _time_matvec(dm, torch, stream, h, xd, reps)
            if nb in yref:
                y = dm.dm_matvec(h, xs[nb])
                r["hmatvec_error_vs_fp64"] = float(np.abs(y - yref[nb]).max() / np.abs(xs[nb]).max())
        dm.dm_destroy(h)
        cfg = dm.dm_config_default(stream=stream.cuda_stream, block_precision=prec, near_mode=dm.DM_NEAR_CACHED,
                                   block_size=16)
        h = dm.dm_create(X, eps=-1.0, alpha=1.0, cfg=cfg)
        dm.dm_compress(h, W["tol"], W["leaf"], W["rank"])
        ts = []
        for _ in range(3):
            ev, V, conv = dm.dm_eigs(h, W["k"], evecs=True, device_out=True)
            ts.append(dm.dm_get_stats(h)["ms_eigs"])
        r["block16_ms_eigs"] = statistics.median(ts)
        r["block16_converged"] = bool(conv)
        e = accuracy_errors(ref, ev, V.cpu().numpy())
        r["block16_max_rel_eigenvalue_error_vs_fp64"] = e["max_rel_eigenvalue_error"]
        r["block16_subspace_angle_rad_vs_fp64"] = e["subspace_angle_rad"]
        dm.dm_destroy(h)
        out[name] = r
    out["note"] = ("at nrhs <= 64 the near product moves 2 nrhs flops per 4 stored bytes, so HBM, not the tensor "
                   "pipe, bounds it; the tensor cores shorten the compute, the split form keeps FP32-level error")
    return out


def scaling_workload_run(dm, torch, stream) -> dict:
    """The paper's evaluation workload of Section 4.2 (a 100k x 100k Gaussian kernel of 6-D
    random points times a 100k x 512 block), here on the diffusion-normalised operator with
    this library's size limits (leaf <= 512, rank <= 256)."""
    import synth

    X = synth.as_f32(synth.gaussian_cloud(100_000, d=6, seed=0))
    res = {"workload": "6-D standard normal cloud N=100000, eps=median sq. distance, alpha=1, leaf 512, "
                       "max rank 256, tol 1e-3, nrhs=512",
           "paper_context": "GOFMM on one 48-core Skylake node (leaf 768, rank 768, tol 1e-3, plain Gaussian "
                            "kernel): compression 13 s (text) / 38.4 s (figure), 100k x 512 evaluation 1.35 s "
                            "(text) / 4.5 s (figure)"}
    g = torch.Generator(device="cuda").manual_seed(4)
    xb = (torch.rand(512, X.shape[0], device="cuda", generator=g) * 2 - 1).t()
    for prec, name in ((dm.DM_PREC_TF32, "tf32"), (dm.DM_PREC_TF32X3, "tf32x3"), (dm.DM_PREC_FP32, "fp32")):
        cfg = dm.dm_config_default(stream=stream.cuda_stream, block_precision=prec, near_mode=dm.DM_NEAR_CACHED)
        t0 = time.perf_counter()
        h = dm.dm_create(X, eps=-1.0, alpha=1.0, cfg=cfg)
        dm.dm_compress(h, 1e-3, 512, 256)
        torch.cuda.synchronize()
        if name == "tf32":
            res["create_compress_s"] = time.perf_counter() - t0
            st = dm.dm_get_stats(h)
            res["ranks"] = {"min": st["rank_min"], "max": st["rank_max"], "mean": round(st["rank_mean"], 2)}
        res[f"matvec_nrhs512_{name}_s"] = _time_matvec(dm, torch, stream, h, xb, 5) / 1e3
        dm.dm_destroy(h)
    return res


def batched_clouds_run(dm, n_clouds: int = 256, slots: int = 8, seed: int = 3) -> dict:
    """Many uneven clouds: n_clouds s-curve / swiss-roll clouds (alternating) with N log-uniform
    in [1000, 32000], top 8 eigenpairs each, max rank 64, tol 1e-5; the leaf size is picked
    per size octave by the autotuner (dm_tune_leaf over {64, 128, 256} on the octave's first
    cloud). Batched: every cloud is created and compressed, then dm_eigs_batch advances all
    their Lanczos steps together (two H-matvec launches and three Gram-Schmidt launches per
    step for all clouds). For comparison the same clouds also go through the request server
    (8 slots build them; their Lanczos steps join its batched solver as they arrive). Reported:
    clouds/s and eigenpairs/s."""
    import numpy as np

    import synth

    Ns = synth.log_uniform_sizes(n_clouds, 1000, 32000, seed=seed)
    clouds = [synth.as_f32(synth.s_curve(int(n), seed=100 + i) if i % 2 == 0 else synth.swiss_roll(int(n), seed=100 + i))
              for i, n in enumerate(Ns)]
    octave = np.floor(np.log2(Ns / 1000.0)).astype(int)
    leaf_of = {}
    t0 = time.perf_counter()
    for o in sorted(set(octave.tolist())):
        i = int(np.where(octave == o)[0][0])
        h = dm.dm_create(clouds[i], eps=-1.0)
        best, _ = dm.dm_tune_leaf(h, 1e-5, 64, 8, candidates=(64, 128, 256))
        dm.dm_destroy(h)
        leaf_of[o] = best
    tune_s = time.perf_counter() - t0
    out = {"workload": f"{n_clouds} clouds (s-curve / swiss roll), N log-uniform in [1000, 32000], top 8, "
                       "max rank 64, tol 1e-5, autotuned leaf",
           "leaf_by_octave": {str(int(1000 * 2 ** o)): leaf_of[o] for o in leaf_of}, "tune_s": tune_s}
    # batched: per-cloud create + compress on 8 host threads (each handle has its own stream;
    # the library calls release the interpreter lock), then one dm_eigs_batch over all clouds
    import concurrent.futures as cf

    def prepare(args):
        X, o = args
        h = dm.dm_create(X, eps=-1.0)
        dm.dm_compress(h, 1e-5, leaf_of[int(o)], 64)
        return h

    for rep in range(2):
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=slots) as ex:
            hs = list(ex.map(prepare, zip(clouds, octave)))
        t1 = time.perf_counter()
        l0 = dm.dm_kernel_launches()
        ev, _, status = dm.dm_eigs_batch(hs, 8, evecs=True)
        t2 = time.perf_counter()
        launches = dm.dm_kernel_launches() - l0
        steps = max(dm.dm_get_stats(h)["lanczos_iters"] for h in hs)
        for h in hs:
            dm.dm_destroy(h)
    ok = int(np.sum(status == dm.DM_OK))
    wall = t2 - t0
    out.update({"wall_s": wall, "create_compress_s": t1 - t0, "eigs_batch_s": t2 - t1,
                "clouds_per_s": n_clouds / wall, "eigenpairs_per_s": 8 * ok / wall,
                "eigs_batch_eigenpairs_per_s": 8 * ok / (t2 - t1), "converged": ok,
                "eigs_batch_launches": int(launches), "lanczos_steps": int(steps),
                "solver": "dm_eigs_batch: single-vector Lanczos per cloud, every cloud's step in the same launches"})
    # the same clouds as independent serving requests
    dm.dm_serve_start(slots=slots, hbm_budget_bytes=150_000_000_000)
    done = {}
    try:
        t0 = time.perf_counter()
        tickets = [dm.dm_submit(X, eps=-1.0, tol=1e-5, leaf_size=leaf_of[int(o)], max_rank=64, k=8,
                                want_vectors=True, seed=0) for X, o in zip(clouds, octave)]
        while len(done) < len(tickets):
            for t in tickets:
                if t not in done:
                    fin, r = dm.dm_poll(t)
                    if fin:
                        done[t] = (r["status"], r["done_ms"] - r["submit_ms"])
            time.sleep(0.0005)
        wall_s = time.perf_counter() - t0
    finally:
        dm.dm_serve_stop()
    ok_s = sum(1 for v in done.values() if v[0] == 0)
    out["via_serving"] = {"wall_s": wall_s, "clouds_per_s": n_clouds / wall_s, "eigenpairs_per_s": 8 * ok_s / wall_s,
                          "converged": ok_s, "slots": slots,
                          "solver": "request server: builds on the slots, single-vector Lanczos steps of every "
                                    "resident request in the batched solver's shared launches"}
    return out


def mnist_workload_run(dm, stream, reps: int = 2) -> dict:
    """The high-dimensional workload: 60,000 MNIST-shaped vectors in R^784 (8-bit quantised,
    ~80% zeros; synthetic stand-in for MNIST), eps = median, leaf 256, rank 128, tol 1e-4,
    top 10; degree passes on the tensor cores (exact BF16 Gram matrix)."""
    import synth

    import torch

    # the points in pinned host memory (the 188 MB copy into the handle is then a DMA at
    # link speed instead of a staged pageable copy)
    X0 = synth.as_f32(synth.mnist_like(60_000, seed=0))
    Xt = torch.empty(X0.shape, dtype=torch.float32, pin_memory=True)
    X = Xt.numpy()
    X[...] = X0
    out = {"workload": "MNIST-shaped N=60000 d=784, eps=median, alpha=1, leaf 256, rank 128, tol 1e-4, top-10",
           "points": "pinned host memory"}
    ts = []
    for _ in range(reps):
        cfg = dm.dm_config_default(stream=stream.cuda_stream)
        t0 = time.perf_counter()
        h = dm.dm_create(X, eps=-1.0, alpha=1.0, cfg=cfg)
        dm.dm_compress(h, 1e-4, 256, 128)
        ev, _, conv = dm.dm_eigs(h, 10, evecs=True, device_out=True)
        ts.append(time.perf_counter() - t0)
        st = dm.dm_get_stats(h)
        dm.dm_destroy(h)
    out.update({"wall_s_median": statistics.median(ts), "eigenpairs_per_s": 10 / statistics.median(ts),
                "phases_ms": {key: round(float(st[key]), 3) for key in
                              ("ms_create", "ms_degrees", "ms_tree", "ms_skeleton", "ms_pack", "ms_eigs")},
                "degree_path": st["degree_path"], "converged": bool(conv), "lanczos_iters": st["lanczos_iters"],
                "ranks": {"min": st["rank_min"], "max": st["rank_max"], "mean": round(st["rank_mean"], 2)},
                "evals_head": [round(float(v), 8) for v in ev[:5]]})
    return out


# ------------------------------------------------------------------ oracle (CPU baseline / reference arm)

def oracle_sample(n: int = WORKLOAD["N"]) -> dict:
    """The FP64 oracle's full pipeline on an n-point s-curve of the same workload; when n is
    below the workload's N, phase times are scaled to it (degrees as N^2, the rest as N log N)."""
    import numpy as np

    import oracle as O
    import synth

    W = WORKLOAD
    X = synth.as_f32(synth.s_curve(n, 0))
    t = {}
    t0 = time.perf_counter()
    eps = O.median_sqdist(X)
    t["median"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    q, dg, s = O.degrees(X, eps, 1.0)
    t["degrees"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    perm, L = O.tree(X, eps, W["leaf"])
    t["tree"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = O.skeletonize(X, eps, s, perm, L, W["tol"], W["rank"])
    t["skeleton"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev, _, it, st = O.lanczos_hmat(X, eps, s, H, W["k"], conv_tol=1e-7)
    t["lanczos"] = time.perf_counter() - t0
    N = W["N"]
    nlog = (N * math.log2(N)) / (n * math.log2(n))
    total = t["median"] + t["degrees"] * (N / n) ** 2 + (t["tree"] + t["skeleton"] + t["lanczos"]) * nlog
    sample_s = sum(t.values())
    if n >= N:
        desc = (f"full FP64 oracle pipeline on the whole {N}-point workload (same generator and parameters; "
                f"{sample_s:.1f} s wall on the host cores, {it} Lanczos steps; no extrapolation)")
    else:
        desc = (f"full FP64 oracle pipeline on a {n}-point s-curve (same generator and parameters; "
                f"{sample_s:.1f} s wall on the host cores, {it} Lanczos steps), phase times scaled to N={N} "
                f"(degrees x (N/n)^2, tree/compression/Lanczos x N log N / n log n)")
    return {"value": W["k"] / total, "unit": UNIT, "cores": O.threads(), "kind": "oracle", "sample": desc,
            "phases_s": {k: round(v, 4) for k, v in t.items()}, "extrapolated_s": round(total, 2)}


def run_reference(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    # warm-up steps (untimed) run the same pipeline on 10,000 points: the host code has no
    # state to warm beyond its first pass, and full-size warm-ups would only lengthen the run.
    # The last one's phase times scaled to the workload predict a full-size step on these cores.
    full_s = ORACLE_FULL_S
    for _ in range(max(1, args.warmup)):
        full_s = oracle_sample(10_000)["extrapolated_s"]
    n_sample = reference_sample_n(args.steps, full_s)
    runs = [oracle_sample(n_sample) for _ in range(args.steps)]
    vals = [r["value"] for r in runs]
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": WORKLOAD["k"] / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"], "N": WORKLOAD["N"], "k": WORKLOAD["k"],
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": runs[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm

def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time for the barrier-bracketed region (every rank passes the
    same collective); the time itself when there is one rank."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(k: int, steps: int, world: int, ms: float) -> float:
    """Eigenpairs per second of the whole job: each of `world` replicas solves `steps`
    problems of k pairs within the slowest rank's `ms`."""
    return k * steps * world / (ms / 1e3)


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def load_traffic() -> dict | None:
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def run_ours(args) -> int:
    import torch

    import paper_2311_06115_gb300 as dm
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dm.load()
    W = dict(WORKLOAD)
    W["N"] = args.n
    X = synth.as_f32(synth.s_curve(W["N"], seed=rank))
    Xd = torch.from_numpy(X).cuda()
    Xh = torch.from_numpy(X).pin_memory()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()  # the library's stream: events below are recorded on it

    def cfg():
        return dm.dm_config_default(profile=1, stream=stream.cuda_stream)

    last = {}

    def step(points, device_out: bool):
        h = dm.dm_create(points, eps=-1.0, alpha=1.0, cfg=cfg())
        dm.dm_compress(h, W["tol"], W["leaf"], W["rank"])
        ev, vec, conv = dm.dm_eigs(h, W["k"], evecs=True, device_out=device_out)
        last["stats"] = dm.dm_get_stats(h)
        last["ev"] = ev
        last["conv"] = conv
        dm.dm_destroy(h)
        return ev, vec

    def timed(points, device_out, steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = dm.dm_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        mv = []
        e0.record(stream)
        for _ in range(steps):
            step(points, device_out)
            st = last["stats"]
            if st["matvec_calls"]:
                mv.append((st["ms_matvec"] / st["matvec_calls"], st["matvec_bytes"]))
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        launches = dm.dm_kernel_launches() - l0
        return ms, launches, mv

    if args.skip_headline:
        out = {}
        for key in (x for x in args.sections.split(",") if x):
            fn = {"accuracy": lambda: accuracy_run(dm, torch, stream, X, W),
                  "precision": lambda: precision_run(dm, torch, stream, X, W),
                  "block_matvec": lambda: block_run(dm, torch, stream, X, W),
                  "block_lanczos": lambda: block_lanczos_run(dm, stream, X, W),
                  "scaling_workload": lambda: scaling_workload_run(dm, torch, stream),
                  "mnist_workload": lambda: mnist_workload_run(dm, stream),
                  "batched_clouds": lambda: batched_clouds_run(dm),
                  "serving": lambda: serve_run(dm, args.serve_requests, args.serve_rate, args.serve_slots,
                                               [int(x) for x in args.serve_dims.split(",")])}[key]
            out[key] = fn()
            if key == "serving" and out[key]["saturated"]:
                sustained = round(0.8 * out[key]["requests_per_s"], 1)
                out["serving_sustained"] = serve_run(dm, max(300, args.serve_requests // 3), sustained,
                                                     args.serve_slots, [int(x) for x in args.serve_dims.split(",")],
                                                     warm=50)
        if rank == 0:
            print(json.dumps({"profiling_only": True, **out}))
        return 0
    for _ in range(args.warmup):
        step(Xd, True)
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches, mv = timed(Xd, True, args.steps)
    clk = clocks.stop()
    # end to end through host buffers (pinned points in, eigenpairs out to host memory)
    for _ in range(max(1, min(args.warmup, 2))):
        step(Xh, False)
    ms_e2e, _, _ = timed(Xh, False, args.steps)
    k = W["k"]
    value = job_throughput(k, args.steps, world, ms)
    e2e_value = job_throughput(k, args.steps, world, ms_e2e)
    st = last["stats"]
    peaks = load_peaks()
    mv_ms = statistics.median([m for m, _ in mv]) if mv else None
    mv_bytes = mv[-1][1] if mv else None
    achieved = (mv_bytes / (mv_ms * 1e-3) / 1e9) if mv_ms else None
    traffic = load_traffic()
    roofline = {"kernel": "H-matvec (leaf_n2s_kernel + tree_kernel + near_cached_kernel chained by programmatic dependent launch; nrhs=1, cached leaf blocks)", "bound": "hbm",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                "traffic": traffic.get("hmatvec_bytes_per_launch") if traffic else None,
                "peak_source": peaks["source"] + " (copy bandwidth, MEASURED_PEAKS.json)",
                "algorithmic_bytes": mv_bytes, "avg_ms": mv_ms}
    # the degree passes (d = 3, CUDA cores): exponentials per second against the MUFU ex2 rate
    # measured by the library's own microbenchmark in this run
    ex2_n, ex2_ms = dm.dm_sfu_peak()
    sfu_peak = ex2_n / (ex2_ms * 1e-3)
    deg_ms = float(st.get("ms_degrees", 0.0))
    deg_ex2 = 2 * W["N"] * (W["N"] + 1) / 2  # two passes over the upper triangle of W (symmetric tiles)
    roofline_degree = {"kernel": "degree_sym_d3_kernel (both degree passes of dm_create, upper tiles of the "
                                 "symmetric W)", "bound": "sfu",
                       "achieved": (deg_ex2 / (deg_ms * 1e-3)) if deg_ms > 0 else None, "peak": sfu_peak,
                       "unit": "ex2/s", "frac": (deg_ex2 / (deg_ms * 1e-3) / sfu_peak) if deg_ms > 0 else None,
                       "algorithmic_ex2": deg_ex2, "avg_ms": deg_ms,
                       "peak_source": "measured: dm_sfu_peak (independent MUFU ex2 chains, 64 warps per SM, "
                                      "CUDA events) in this run",
                       "peak_per_sm_clock": (sfu_peak / (torch.cuda.get_device_properties(local).multi_processor_count
                                                          * clk["sm_mhz"] * 1e6)) if clk.get("sm_mhz") else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 sums and tridiagonal)", "data": "synthetic",
            "config": {"workload": W["workload"] if W["N"] == WORKLOAD["N"] else f"s-curve N={W['N']}",
                       "N": W["N"], "k": k, "leaf": W["leaf"], "max_rank": W["rank"], "tol": W["tol"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "per-step working set (leaf blocks + Krylov basis) exceeds L2"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": W["N"] * W["d"] * 4,
                    "d2h_bytes_per_step": k * 8 + W["N"] * k * 4},
            "gpu_launches": int(launches), "roofline": roofline, "roofline_degree": roofline_degree, "clocks": clk,
            "phases_ms": {key: round(float(st[key]), 3) for key in
                          ("ms_create", "ms_degrees", "ms_tree", "ms_skeleton", "ms_pack", "ms_eigs")},
            "lanczos_iters": st["lanczos_iters"], "converged": bool(last["conv"]),
            "ranks": {"min": st["rank_min"], "max": st["rank_max"], "mean": round(st["rank_mean"], 2)},
            "evals_head": [round(float(v), 8) for v in last["ev"][:5]]}
    if world == 1 and not args.no_block:
        wanted = set(x for x in args.sections.split(",") if x)
        for key, fn in (("precision", lambda: precision_run(dm, torch, stream, X, W)),
                        ("block_matvec", lambda: block_run(dm, torch, stream, X, W)),
                        ("block_lanczos", lambda: block_lanczos_run(dm, stream, X, W)),
                        ("scaling_workload", lambda: scaling_workload_run(dm, torch, stream)),
                        ("mnist_workload", lambda: mnist_workload_run(dm, stream)),
                        ("batched_clouds", lambda: batched_clouds_run(dm))):
            if key not in wanted:
                continue
            try:
                line[key] = fn()
            except Exception as exc:  # a failed side measurement must not hide the headline line
                line[key] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and "accuracy" in set(x for x in args.sections.split(",") if x):
        try:
            line["accuracy"] = accuracy_run(dm, torch, stream, X, W)
        except Exception as exc:
            line["accuracy"] = {"error": f"{type(exc).__name__}: {exc}"}
    if args.serve_requests > 0 and world == 1:
        dims = [int(x) for x in args.serve_dims.split(",")]
        line["serving"] = serve_run(dm, args.serve_requests, args.serve_rate, args.serve_slots, dims)
        if line["serving"]["saturated"]:
            # the offered rate exceeds capacity: latency there is backlog; measure it again at a
            # rate the server sustains (80% of the completion rate just measured)
            sustained = round(0.8 * line["serving"]["requests_per_s"], 1)
            line["serving_sustained"] = serve_run(dm, max(300, args.serve_requests // 3), sustained,
                                                  args.serve_slots, dims, warm=50)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        line["cpu_baseline"] = oracle_sample()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main() -> int:
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
