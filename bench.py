#!/usr/bin/env python
"""Benchmark: MRHS multigrid solves per second to a true residual of 1e-10.

Workload (one step = one MRHS solve of the whole RHS block):
  24^3 x 64 lattice, antiperiodic t, U = exp(i 0.25 H) with seeded Gaussian
  traceless Hermitian H, c_sw = 1, mass below, three-level MG (4^4 then 2^4
  aggregates, 32 chirally split null vectors each, even-odd fine smoother),
  nRHS = 48 Gaussian
  sources, outer FP64 FGMRES (float-float Arnoldi products, FP64 residual
  gate), FP32 inner FGMRES + V-cycle, FP16 tensor-core
  coarse stencil and intergrid transfers, V-cycle replayed as a CUDA graph,
  tol 1e-10.
Setup (null vectors, Galerkin) runs before the timed region and is reported
separately.  The line also carries the plain one-RHS-at-a-time solver (FP32
coarse stencil on CUDA cores, no graphs) on the same GPU, the fine-stencil
roofline, the end-to-end number with host buffers, a continuous-batching
serving run (p50 / p99 latency), and the oracle timed on the host cores as
the CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --case stencil|schur|intergrid|blas   (small cases for ncu captures)
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(dims=(24, 24, 24, 64), eps=0.25, gauge_seed=1301, source_seed=2301, mass=-0.13, csw=1.0,
                nrhs=48, tol=1e-10, n_levels=3, blocks=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[32, 32])
MG_PARAMS = dict(setup_sweeps=6, setup_m=8, smooth_m=3, coarse_m=14, coarse_cycles=1, inter_m=4, inner_m=5,
                 inner_max_iters=200, inner_tol=1e-5, outer_m=4, max_outer_iters=30, smoother_evenodd=1)
# the kernel with the largest share of a timed solve in the profiler's launch list (the even-odd
# hopping kernel of the fine smoother's Schur operator), and the full-lattice fine stencil; the
# names are the kernel timer's, which cover the paired (k_eo_x2, k_dslash_x2) and the
# one-RHS-per-thread (k_eo_r1, k_dslash_r1) forms
DOMINANT_KERNEL = "k_eo_x2"
FINE_STENCIL_KERNEL = "k_dslash_x2"
WORKLOAD_NAME = ("wilson-clover MG solve 24^3x64 antiperiodic, U=exp(i0.25H), c_sw=1, 3 levels "
                 "(4^4, 2^4 aggregates, 32 null vectors, even-odd fine smoother), nRHS=48, tol 1e-10")
# the CPU baseline / reference arm: the oracle's FP64 MG-FGMRES with the
# benchmarked structure (3 levels, 4^4 then 2^4 aggregates, 32 null vectors per
# level, even-odd fine post-smoother, the cycle parameters of MG_PARAMS) on 8^4,
# the smallest lattice both aggregations divide, of the same gauge recipe and
# mass; its time per RHS is scaled to the workload by the volume ratio
ORACLE_SAMPLE = dict(dims=(8, 8, 8, 8))


def volume(d):
    return d[0] * d[1] * d[2] * d[3]


# ------------------------------------------------------------------ helpers
def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2211_13719_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


STENCIL_SOURCES = ("dirac.cu", "pair.cuh", "spin.cuh")


def profiled_traffic(name):
    """dram bytes per launch from a committed ncu summary, if the kernel sources are unchanged."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("source_hash") == source_hash(*STENCIL_SOURCES):
            return rec
    except Exception:
        pass
    return None


# -------------------------------------------------------------- N replicas
def max_over_ranks(t, world, device):
    """The job time: the slowest rank's time (all-reduce MAX over the ranks)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(nrhs_per_rank, steps, world, t_job):
    """Whole-job solves/s: every rank (replica) solves its own nrhs_per_rank RHS per step."""
    return nrhs_per_rank * steps * world / t_job


def replica_source_seed(w, rank):
    """Each replica draws its own sources."""
    return w["source_seed"] + 1000 * rank


# --------------------------------------------------------------- oracle arm
def oracle_sample_solve(steps: int, warmup: int):
    """Time the oracle's FP64 MG-FGMRES on the sample lattice (one RHS per step)."""
    import numpy as np

    import synth
    from oracle import mg as omg
    w = WORKLOAD
    dims = ORACLE_SAMPLE["dims"]
    U = synth.gauge_exp(dims, w["eps"], w["gauge_seed"])
    p = oracle_workload_params()
    V = volume(dims)
    d1 = tuple(L // w["blocks"][0][mu] for mu, L in enumerate(dims))
    t0 = time.perf_counter()
    levels = omg.build_hierarchy(U, dims, w["mass"], w["csw"], p,
                                 [synth.gaussian_field(V, 12, w["nvec"][0], 7),
                                  synth.gaussian_field(volume(d1), 64, w["nvec"][1], 8)])
    setup_s = time.perf_counter() - t0
    times = []
    for i in range(warmup + steps):
        b = synth.gaussian_field(V, 12, 1, w["source_seed"] + i)
        t0 = time.perf_counter()
        x, hist = omg.solve(levels, b, p)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
        assert np.all(hist[-1] <= w["tol"])
    mean = sum(times) / len(times)
    scale = V / volume(w["dims"])
    return {"value": scale / mean, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle FP64 MG-FGMRES, 1 RHS per step on {dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} "
                       f"(same gauge recipe and mass; the benchmarked structure: 3 levels, 4^4 then 2^4 "
                       f"aggregates, 32 null vectors per level, even-odd fine smoother), {mean:.2f} s per "
                       f"solve (setup {setup_s:.1f} s, not counted), scaled by the volume ratio "
                       f"{V}/{volume(w['dims'])}"),
            "seconds_per_sample_solve": mean, "sample_setup_s": setup_s}


def oracle_workload_params():
    """The oracle's MGParams for the benchmarked structure (WORKLOAD, MG_PARAMS)."""
    from oracle import mg as omg
    w = WORKLOAD
    return omg.MGParams(blocks=w["blocks"], nvec=w["nvec"], setup_sweeps=MG_PARAMS["setup_sweeps"],
                        setup_m=MG_PARAMS["setup_m"], smooth_m=MG_PARAMS["smooth_m"],
                        coarse_m=MG_PARAMS["coarse_m"], coarse_cycles=1, inter_m=MG_PARAMS["inter_m"],
                        outer_m=MG_PARAMS["inner_m"], tol=w["tol"], smoother_evenodd=True)


def oracle_in_subprocess(steps=1, warmup=0):
    """Run the oracle timing on one host thread in a fresh process (spawned after CUDA use)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample_solve(%d, %d)))" % (ROOT, steps, warmup))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if p.returncode != 0:
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "failed: " +
                p.stderr.strip().splitlines()[-1] if p.stderr.strip() else "failed"}
    return json.loads(p.stdout.strip().splitlines()[-1])


# ------------------------------------------------------- oracle timing table
# The CPU baseline items: the oracle (plain numpy, FP64) timed on the host
# cores.  Fine apply on the 24^4 Haar lattice (c_sw = 1, m = -0.2); coarse
# 9-point apply on 6^4 with nc = 64 (random links of the Galerkin shape: the
# values do not change the work); the small plain solve (8^4, eps 0.4,
# m = -0.2, 4 RHS, 2 levels, 4^4 aggregates, 8 null vectors); and one RHS of
# the benchmarked 3-level / 32-vector structure on 8^4, the smallest lattice
# its 4^4 and 2^4 aggregations divide (setup reported separately).
def oracle_table_items(which=None):
    import numpy as np

    import synth
    from oracle import coarse as oc, mg as omg, wilson as ow
    out = {}

    def timed(fn, reps=1):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) / reps

    if which in (None, "fine"):
        dims = (24, 24, 24, 24)
        U = synth.gauge_haar(dims, 1101)
        C = ow.clover_term(U, dims, 1.0)
        V = volume(dims)
        for n in (1, 12, 64):
            psi = synth.gaussian_field(V, 12, n, 2101)
            t = timed(lambda: ow.apply_D(U, C, psi, dims, -0.2))
            out[f"fine_apply_24^4_n{n}_s"] = t
            out[f"fine_apply_24^4_n{n}_GBs"] = V * (576 + 192 * n) / t / 1e9
            del psi
        del U, C
    if which in (None, "coarse"):
        cd = (6, 6, 6, 6)
        Vc = volume(cd)
        rng = np.random.default_rng(1201)
        A = (rng.standard_normal((Vc, 9, 64, 64)) + 1j * rng.standard_normal((Vc, 9, 64, 64))) / 64
        for n in (12, 48):
            phi = synth.gaussian_field(Vc, 64, n, 2201)
            t = timed(lambda: oc.apply_coarse(A, phi, cd), reps=2)
            out[f"coarse_apply_6^4_nc64_n{n}_s"] = t
        del A
    if which in (None, "c0"):
        dims = (8, 8, 8, 8)
        U = synth.gauge_exp(dims, 0.4, 1001)
        p = omg.MGParams(blocks=[(4, 4, 4, 4)], nvec=[8], setup_sweeps=4, setup_m=8, smooth_m=4, coarse_m=16,
                         coarse_cycles=2, outer_m=8, tol=1e-10)
        t0 = time.perf_counter()
        levels = omg.build_hierarchy(U, dims, -0.2, 1.0, p, [synth.gaussian_field(volume(dims), 12, 8, 7)])
        out["c0_setup_s"] = time.perf_counter() - t0
        b = synth.gaussian_field(volume(dims), 12, 4, 2001)
        t0 = time.perf_counter()
        x, hist = omg.solve(levels, b, p)
        out["c0_solve_4rhs_s"] = time.perf_counter() - t0
        out["c0_outer_cycles"] = len(hist) - 1
        out["c0_max_rel_residual"] = float(np.max(hist[-1]))
    if which in (None, "c3"):
        w = WORKLOAD
        dims = (8, 8, 8, 8)
        U = synth.gauge_exp(dims, w["eps"], w["gauge_seed"])
        d1 = tuple(L // 4 for L in dims)
        p = oracle_workload_params()
        t0 = time.perf_counter()
        levels = omg.build_hierarchy(U, dims, w["mass"], w["csw"], p,
                                     [synth.gaussian_field(volume(dims), 12, 32, 7),
                                      synth.gaussian_field(volume(d1), 64, 32, 8)])
        out["c3_structure_8^4_setup_s"] = time.perf_counter() - t0
        b = synth.gaussian_field(volume(dims), 12, 1, w["source_seed"])
        t0 = time.perf_counter()
        x, hist = omg.solve(levels, b, p)
        t = time.perf_counter() - t0
        out["c3_structure_8^4_solve_1rhs_s"] = t
        out["c3_structure_8^4_outer_cycles"] = len(hist) - 1
        out["c3_per_rhs_scaled_to_24^3x64_s"] = t * volume(w["dims"]) / volume(dims)
    return out


def oracle_table(threads):
    """Run oracle_table_items in a fresh process with `threads` BLAS / OpenMP threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads), CUDA_VISIBLE_DEVICES="")
    res = {"threads": threads, "nproc": os.cpu_count()}
    for item in ("fine", "coarse", "c0", "c3"):
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_table_items(%r)))" % (ROOT, item))
        p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=7200)
        if p.returncode != 0:
            res[item] = "failed: " + (p.stderr.strip().splitlines() or ["?"])[-1]
        else:
            res.update(json.loads(p.stdout.strip().splitlines()[-1]))
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.perf_counter()
    res = oracle_in_subprocess(args.steps, args.warmup)
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": "MG solves/s at 1e-10", "value": res["value"], "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (res.get("seconds_per_sample_solve") or 0) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample": ORACLE_SAMPLE["dims"]},
        "cpu_baseline": {"value": res["value"], "unit": "solves/s", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": res["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def make_params(mrhs, n_max, coarse_precision, use_graph, **over):
    p = mrhs.mrhs_mg_default_params()
    w = WORKLOAD
    p.n_levels = w["n_levels"]
    for l, b in enumerate(w["blocks"]):
        for mu in range(4):
            p.block[l][mu] = b[mu]
    for l, nv in enumerate(w["nvec"]):
        p.n_vec[l] = nv
    for k, v in dict(MG_PARAMS, **over).items():
        setattr(p, k, v)
    p.max_rhs = n_max
    p.coarse_precision = coarse_precision
    p.use_graph = use_graph
    p.seed = 4242
    return p


def smoother_params(args):
    """MG parameter overrides of the --smoother and --coarse-smoother choices."""
    out = {}
    if args.smoother == "sap":
        out = dict(smoother_sap=1, smoother_evenodd=0, sap_mr=args.sap_mr, sap_cycles=args.sap_cycles)
    elif args.smoother == "gmres":
        out = dict(smoother_sap=0, smoother_evenodd=0)
    if args.coarse_smoother == "evenodd":
        out["coarse_smoother_evenodd"] = 1
    if args.coarse_solver == "gcrodr":
        out.update(coarse_solver=1, coarse_recycle=args.coarse_recycle)
        if args.coarse_m:
            out["coarse_m"] = args.coarse_m
    out["coarse_fused"] = args.coarse_fused
    return out


def gauge_field(w):
    import numpy as np

    import synth
    # keyed on the generator's source, so a change to synth never reuses a stale field
    with open(os.path.join(ROOT, "synth", "fields.py"), "rb") as f:
        gen = hashlib.sha256(f.read()).hexdigest()[:12]
    cache = f"/tmp/mrhs_bench_gauge_{w['dims']}_{w['eps']}_{w['gauge_seed']}_{gen}.npy".replace(" ", "")
    if os.path.exists(cache):
        try:
            return np.load(cache)
        except Exception:
            pass
    U = synth.gauge_exp(w["dims"], w["eps"], w["gauge_seed"])
    try:
        np.save(cache, U)
    except Exception:
        pass
    return U


SERVE_SMALL = dict(dims=(16, 16, 16, 32), gauge_seed=1402)


def run_serving(mrhs, mg_big, w, saturated, args, torch, np, load=None, nreq=None):
    """Poisson arrivals of 1..12-source requests, 50/50 over two resident
    hierarchies (the 24^3x64 one and a 16^3x32 one of the same recipe), at
    `load` times the measured saturated solves/s; p50 / p99 latency, and the
    time each request waited for admission (queue) against the time it then
    spent in the batched solve."""
    load = args.serve_load if load is None else load
    nreq = args.serve_requests if nreq is None else nreq
    import synth
    dims_s = SERVE_SMALL["dims"]
    Us = synth.gauge_exp(dims_s, w["eps"], SERVE_SMALL["gauge_seed"])
    lat_s = mrhs.mrhs_create_lattice(dims_s, -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat_s, Us)
    mrhs.mrhs_build_clover(lat_s, w["mass"], w["csw"])
    mg_s = mrhs.mrhs_setup_mg(lat_s, make_params(mrhs, w["nrhs"], mrhs.MRHS_FP16, 1))
    srv = mrhs.mrhs_server_create(max_queue=4096, hbm_reserve_gb=2.0)
    try:
        cids = [mrhs.mrhs_server_add_config(srv, mg_big, w["nrhs"]),
                mrhs.mrhs_server_add_config(srv, mg_s, w["nrhs"])]
        vols = [volume(w["dims"]), volume(dims_s)]
        rng = np.random.default_rng(3001)
        # sources drawn once per config and reused (values do not affect the schedule): a request of
        # nr sources takes the first V*12*nr values of its config's pool as its [V][12][nr] array,
        # so no request copies or holds a source buffer of its own
        pool = [synth.gaussian_field(vols[c], 12, 12, 2401 + c).reshape(-1) for c in range(2)]
        # offered load in requests/s: fraction of the RHS throughput, mean 6.5 RHS per request,
        # the small config costs about its volume ratio of a big solve
        mean_cost = 0.5 * (1.0 + vols[1] / vols[0]) * 6.5
        rate = load * saturated / mean_cost
        pending = {}  # request id -> (config, nr, solution buffer), until the server reports completion
        lat, qt, ok, solves, done = [], [], 0, 0, 0
        equiv = 0.0  # solves weighted by volume relative to the big config (the unit of the offered load)

        def collect():
            nonlocal ok, solves, done, equiv
            for rid in list(pending):
                st, rs = mrhs.mrhs_poll(srv, rid)
                if st == mrhs.MRHS_PENDING:
                    continue
                c, nr, _x = pending.pop(rid)  # the solution buffer is released here
                lat.append(rs.latency_s)
                qt.append(rs.queue_s)
                done += 1
                if st == mrhs.MRHS_OK:
                    ok += 1
                    solves += nr
                    equiv += nr * vols[c] / vols[0]

        t0 = time.perf_counter()
        t_next = t0
        for i in range(nreq):
            t_next += rng.exponential(1.0 / rate)
            while time.perf_counter() < t_next:
                time.sleep(0.0005)
            c = int(rng.integers(0, 2))
            nr = int(rng.integers(1, 13))
            b = pool[c][:vols[c] * 12 * nr].reshape(vols[c], 12, nr)
            x = np.empty_like(b)
            rid = mrhs.mrhs_submit(srv, cids[c], b, x, nr, w["tol"])
            pending[rid] = (c, nr, x)
            collect()
        mrhs.mrhs_server_drain(srv)
        wall = time.perf_counter() - t0
        collect()
        lat_ms = np.array(lat) * 1e3
        q_ms = np.array(qt) * 1e3
        s_ms = lat_ms - q_ms
        return {"requests": done, "completed_ok": ok, "solves": solves, "wall_s": wall,
                "solves_per_s": solves / wall, "offered_load": load,
                "big_equivalent_solves_per_s": equiv / wall,
                "offered_big_equivalent_solves_per_s": load * saturated,
                "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "queue_p50_ms": float(np.percentile(q_ms, 50)), "queue_p99_ms": float(np.percentile(q_ms, 99)),
                "in_solve_p50_ms": float(np.percentile(s_ms, 50)), "in_solve_p99_ms": float(np.percentile(s_ms, 99)),
                "memory_deferred_admissions": mrhs.mrhs_server_memory_waits(srv),
                "configs": [w["dims"], dims_s], "slots_per_config": w["nrhs"],
                "arrivals": "Poisson, seed 3001, 1..12 sources per request, 50/50 configs"}
    finally:
        mrhs.mrhs_server_destroy(srv)
        mrhs.mrhs_destroy_mg(mg_s)
        mrhs.mrhs_destroy_lattice(lat_s)


def autotune_summary(mrhs):
    out = []
    for e in mrhs.mrhs_tune_entries():
        d = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in e.items()}
        if e["kernel"] in ("k_dots_norm", "k_norm2"):
            dims = e["dims"]
            d = {"kernel": e["kernel"], "rows": dims[0] + (dims[1] << 30), "k": dims[2], "nrhs": e["nrhs"],
                 "variant": e["variant"], "rows_per_thread": (4, 16, 64)[e["variant"]],
                 "nvariants": e["nvariants"], "best_ms": d["best_ms"], "default_ms": d["default_ms"]}
        elif e["kernel"] == "k_coarse_tc":
            d["ring_stages"] = (3, 2, 4)[e["variant"]]
        out.append(d)
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2211_13719_gb300 import build as _build
    from paper_2211_13719_gb300 import mrhs

    torch.cuda.set_device(local_rank)
    dev = torch.cuda.current_device()
    if rank == 0:
        _build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        _build.build()
    w = dict(WORKLOAD)
    if args.nrhs:
        w["nrhs"] = args.nrhs
    n = w["nrhs"]
    dims = w["dims"]
    V = volume(dims)
    U = gauge_field(w)
    lat = mrhs.mrhs_create_lattice(dims, -1, dev)
    mrhs.mrhs_load_gauge(lat, U)
    mrhs.mrhs_build_clover(lat, w["mass"], w["csw"])
    del U
    t0 = time.perf_counter()
    mg = mrhs.mrhs_setup_mg(lat, make_params(mrhs, n, mrhs.MRHS_FP16, 1, **smoother_params(args)))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    gen = torch.Generator(device="cuda")
    gen.manual_seed(replica_source_seed(w, rank))
    b = torch.randn((V, 12, n), dtype=torch.complex128, device="cuda", generator=gen)
    x = torch.zeros_like(b)
    rel = np.zeros(n)
    stream = torch.cuda.current_stream()

    def step():
        x.zero_()
        status, st = mrhs.mrhs_solve(mg, b, x, n, w["tol"], rel, stream=stream)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = mrhs.mrhs_kernel_launch_count()
    stats = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # CUDA events around the dominant kernel's launches, on the stream it runs on
    mrhs.mrhs_kernel_timer_start(FINE_STENCIL_KERNEL)
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    k_ms, k_timed, k_captured = mrhs.mrhs_kernel_timer_stop()
    launches = mrhs.mrhs_kernel_launch_count() - launches0
    t_dev = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world, "cuda")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    max_rel = float(max(s.max_rel_residual for s in stats))
    value = job_throughput(n, args.steps, world, t_dev)

    extra = {}
    if rank == 0:
        # --- end to end through the C ABI with host buffers (pinned), copies inside the timed region.
        # Every step uploads its sources and downloads its solution; uploads and downloads run
        # on two copy streams of their own (separate copy engines) into double-buffered device
        # fields, so step k+1's upload and step k - 1's download overlap step k's solve
        # (mrhs_solve returns when its solve is complete); only the first upload and the last
        # download are exposed.
        ke = max(2, min(args.steps, 8))
        bh = [b.cpu().pin_memory() for _ in range(2)]
        xh = [torch.empty_like(bh[0]).pin_memory() for _ in range(2)]
        bd = [b, torch.empty_like(b)]
        xd = [x, torch.empty_like(x)]
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_out = [torch.cuda.Event(), torch.cuda.Event()]
        ev_read = [torch.cuda.Event(), torch.cuda.Event()]
        # the copy rates alone (one upload, one download of a step's field), for context; the
        # first download into fresh page-locked memory also pays for touching its pages, so both
        # download buffers are written once before the timed loop (as in a running pipeline)
        torch.cuda.synchronize()
        rates = {}
        for name, dst, src in (("h2d_GBs", bd[1], bh[0]), ("d2h_first_touch_GBs", xh[0], bd[0]),
                               ("d2h_GBs", xh[0], bd[0]), ("d2h_first_touch_buffer2_GBs", xh[1], bd[0])):
            t0c = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            rates[name] = round(src.numel() * src.element_size() / (time.perf_counter() - t0c) / 1e9, 1)
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        with torch.cuda.stream(up):
            bd[0].copy_(bh[0], non_blocking=True)
            ev_in[0].record(up)
        for k in range(ke):
            i = k % 2
            stream.wait_event(ev_in[i])
            if k + 1 < ke:
                # buffer 1 - i was last read by step k - 1's solve, which has completed
                with torch.cuda.stream(up):
                    up.wait_event(ev_out[1 - i])
                    bd[1 - i].copy_(bh[1 - i], non_blocking=True)
                    ev_in[1 - i].record(up)
            # x buffer i was last read by step k - 2's download
            stream.wait_event(ev_read[i])
            with torch.cuda.stream(stream):
                xd[i].zero_()
            mrhs.mrhs_solve(mg, bd[i], xd[i], n, w["tol"], rel, stream=stream)
            ev_out[i].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_out[i])
                xh[i].copy_(xd[i], non_blocking=True)
                ev_read[i].record(down)
        torch.cuda.synchronize()
        te = time.perf_counter() - te0
        bytes_io = V * 12 * n * 16
        extra["e2e"] = {"value": n * ke / te, "unit": "solves/s", "h2d_bytes_per_step": bytes_io,
                        "d2h_bytes_per_step": bytes_io, "steps": ke,
                        "copies": ("pinned host buffers, upload and download streams of their own, "
                                   "double-buffered device fields"), "copy_rates_alone": rates}
        del bd[1], xd[1]
        # --- component breakdown (one profiled solve, eager V-cycle): the paper's Sec. 8 table
        # (reported from the solve stats of the timed steps)
        s0 = stats[-1]
        extra["per_solve"] = {"outer_iters": s0.outer_iters, "inner_iters": s0.inner_iters, "vcycles": s0.vcycles,
                              "seconds": s0.seconds, "max_rel_residual": max_rel}
        extra["setup_s"] = setup_s
        extra["setup_phases_ms"] = {
            f"level{l}->{l + 1}": dict(zip(("null_vectors", "orthonormalise", "galerkin", "tc_prepare"),
                                           [round(v, 2) for v in mrhs.mrhs_mg_setup_times(mg, l)]))
            for l in range(w["n_levels"] - 1)}
        fi = mrhs.mrhs_coarsest_fused_info(mg)
        extra["coarsest_persistent_kernel"] = {"in_use": bool(fi[0]), "resident_ctas": fi[1],
                                               "coarsest_sites": fi[2]}
        # --- rooflines.  The dominant kernel of a timed solve in the profiler's launch list is the
        # even-odd hopping kernel k_eo_x2 (the Schur operator D_hat = C_oo - 1/4 H_oe C_ee^-1 H_eo of the
        # fine smoother: one C^-1 H launch and one C - 1/4 H launch over V/2 output sites each).  Its
        # launches in the timed region are replayed from the V-cycle graph, where events cannot bracket
        # them, so it is timed with CUDA events on the solver stream around standalone D_hat
        # applications of the same size right after the timed region (half fields of 2 GB: larger
        # than L2).  The full-lattice fine stencil k_dslash_x2 is timed live in the timed region.
        peak, peak_kind = read_peaks()

        def per_call(fn, reps=20):
            for _ in range(3):
                fn()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(reps):
                fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            return ev0.elapsed_time(ev1) * 1e-3 / reps

        a = torch.randn((V, 12, n), dtype=torch.complex64, device="cuda", generator=gen)
        o = torch.empty_like(a)
        t_alone = per_call(lambda: mrhs.mrhs_apply_D(lat, a, o, n, mrhs.MRHS_FP32, stream))
        t_k = k_ms * 1e-3 / k_timed if k_timed else t_alone
        alg = V * (576 + 192 * n)
        tr = profiled_traffic("dslash_fp32_traffic.json")
        extra["roofline_fine_stencil"] = {
            "bound": "hbm", "achieved": alg / t_k / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg / t_k / 1e9 / peak, "traffic": (tr["dram_bytes_per_launch"] if tr else None),
            "kernel": f"{FINE_STENCIL_KERNEL} (fp32 full-lattice fine stencil D; default variant: the "
                      f"one-RHS-per-thread form k_dslash_r1), "
                      f"{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}, nRHS={n}",
            "algorithmic_bytes_per_launch": alg, "bytes_per_site": f"576 + 192 n = {576 + 192 * n}",
            "ms_per_launch": t_k * 1e3,
            "timing": (f"CUDA events on the solver stream around its {k_timed} launches made outside CUDA "
                       f"graphs in the timed region" if k_timed else "timed alone (no launch in the timed region)"),
            "ms_per_launch_alone": t_alone * 1e3,
            "peak_source": f"{peak_kind} HBM copy bandwidth (burst: the kernel is timed per launch)"}
        del a, o
        ah = torch.randn((V // 2, 12, n), dtype=torch.complex64, device="cuda", generator=gen)
        oh = torch.empty_like(ah)
        mrhs.mrhs_kernel_timer_start(DOMINANT_KERNEL)
        t_dhat = per_call(lambda: mrhs.mrhs_apply_schur(lat, ah, oh, n, stream))
        eo_ms, eo_timed, _ = mrhs.mrhs_kernel_timer_stop()
        t_eo = eo_ms * 1e-3 / eo_timed
        # per D_hat: two launches over V/2 output sites; per output site 8 links (4 forward at the
        # site, 4 backward at its neighbours: every link of the lattice once) 576 B, the 6x6 blocks of
        # C^-1 or C 288 B, the 8 neighbour spinors counted once 96 n B, out 96 n B, and for C - 1/4 H
        # the site's own spinor 96 n B: (1728 + 480 n) B per output site and D_hat
        alg_dhat = (V // 2) * (1728 + 480 * n)
        alg_eo = alg_dhat / 2
        tre = profiled_traffic("eo_fp32_traffic.json")
        extra["roofline"] = {
            "bound": "hbm", "achieved": alg_eo / t_eo / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg_eo / t_eo / 1e9 / peak, "traffic": (tre["dram_bytes_per_launch"] if tre else None),
            "kernel": f"{DOMINANT_KERNEL} (fp32 even-odd hopping kernel, both launches of the Schur operator "
                      f"D_hat; default variant: the one-RHS-per-thread form k_eo_r1), "
                      f"{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}, nRHS={n}",
            "algorithmic_bytes_per_launch": alg_eo,
            "bytes_per_output_site": f"per D_hat (2 launches) 1728 + 480 n = {1728 + 480 * n}",
            "ms_per_launch": t_eo * 1e3, "ms_per_dhat": t_dhat * 1e3,
            "timing": (f"CUDA events on the solver stream around {eo_timed} launches of standalone D_hat "
                       f"applications (V/2 x 12 x {n} half fields) after the timed region; inside it the "
                       f"kernel runs from the V-cycle CUDA graph"),
            "peak_source": f"{peak_kind} HBM copy bandwidth (burst: the kernel is timed per launch)"}
        del ah, oh
        # --- plain solver: one RHS at a time, FP32 coarse stencil on CUDA cores, no graphs
        if not args.no_plain:
            mgp = mrhs.mrhs_setup_mg(lat, make_params(mrhs, 1, mrhs.MRHS_FP32, 0))
            b1 = b[:, :, :1].contiguous()
            x1 = torch.zeros_like(b1)
            rel1 = np.zeros(1)
            mrhs.mrhs_solve(mgp, b1, x1, 1, w["tol"], rel1, stream=stream)  # warm-up
            kp = args.plain_solves
            tp0 = time.perf_counter()
            for i in range(kp):
                b1.copy_(b[:, :, i:i + 1])
                x1.zero_()
                mrhs.mrhs_solve(mgp, b1, x1, 1, w["tol"], rel1, stream=stream)
            torch.cuda.synchronize()
            tp = time.perf_counter() - tp0
            plain = kp / tp
            extra["plain"] = {"value": plain, "unit": "solves/s", "solves_timed": kp,
                              "ratio_mixed_batched_over_plain": value / world / plain,
                              "desc": "same MG, nRHS=1, FP32 coarse stencil on CUDA cores, no CUDA graphs, FP64 outer"}
            mrhs.mrhs_destroy_mg(mgp)
        # --- serving: continuous batching over two resident configurations
        if args.serve_requests > 0:
            extra["serving"] = run_serving(mrhs, mg, w, value / world, args, torch, np)
        # --- CPU baseline: the oracle on one host thread, bounded sample
        if not args.no_cpu:
            extra["cpu_baseline"] = oracle_in_subprocess(1, 0)
        extra["clocks"] = clk.summary()
        extra["gpu_launches"] = launches
        # the autotuner's choices, made in the warm-up steps: visit orders of the FP32 fine stencils,
        # ring depth of the tensor-core coarse stencil per level, grids of the batched reductions per
        # field size (their key holds rows = dims[0] + 2^30 dims[1], k = dims[2])
        extra["autotune"] = autotune_summary(mrhs)
        line = {
            "metric": "MG solves/s at 1e-10", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+df64+f32+f16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "nrhs_per_gpu": n, "lattice": "x".join(map(str, dims)),
                       "mass": w["mass"], "csw": w["csw"], "parallelism": f"replicas x{world}",
                       "smoother": args.smoother + (f" (SAP {args.sap_cycles} cycle(s), {args.sap_mr} MR steps, "
                                                    f"4^4 blocks)" if args.smoother == "sap" else ""),
                       "coarse_smoother": args.coarse_smoother,
                       "coarse_solver": args.coarse_solver + (f" (m {args.coarse_m or MG_PARAMS['coarse_m']}, "
                                                              f"k {args.coarse_recycle})"
                                                              if args.coarse_solver == "gcrodr" else "")
                                        + (" (persistent kernel)" if args.coarse_fused and args.coarse_solver == "gmres"
                                           else ""),
                       "l2": "inputs larger than L2 (FP64 fields of 8 GB)"},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    mrhs.mrhs_destroy_mg(mg)
    mrhs.mrhs_destroy_lattice(lat)


# ------------------------------------------------------- profiling cases
def run_case(name, reps, args=None):
    """Small launches of one kernel family, for ncu captures (a few GB on the device).

    stencil:   FP32 fine operator, 24^4 lattice, 48 RHS
    stencil-sweep: FP32 fine operator, 24^4 lattice, nRHS 1 .. 64
    schur:     even-odd hop and Schur operator (FP32), 24^4 lattice, 48 RHS
    intergrid: tensor-core restriction + prolongation, 16^4 lattice, 4^4 aggregates, 32 vectors, 48 RHS
    blas:      the FP32 batched multi-dot and linear combination, 16^4 x 12 rows (--blas-rows), 48 RHS, 4 vectors
    coarsest:  the coarsest GMRES(14) solve at 3^3x8 sites, nc = 64, 48 RHS (small 2-level hierarchy), the
               persistent kernel and the launch-per-operation path
    Prints one JSON line with the CUDA-event time per launch."""
    import numpy as np
    import torch

    from paper_2211_13719_gb300 import build as _build
    from paper_2211_13719_gb300 import mrhs
    import synth

    _build.build()
    n = 48
    stream = torch.cuda.current_stream()

    def ev(fn):
        for _ in range(2):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"case": name, "nrhs": n, "reps": reps}
    if name == "blas":
        rows = args.blas_rows
        k = 4
        basis = torch.randn((k + 1, rows, n), dtype=torch.complex64, device="cuda")
        h = torch.empty((k + 1, n), dtype=torch.complex128, device="cuda")
        out["rows"] = rows
        out["ms_multi_dot_k4"] = ev(lambda: mrhs.mrhs_blas_multi_dot(basis, k, basis[k], rows, n, mrhs.MRHS_FP32, h))
        out["GBs_multi_dot_k4"] = (k + 1) * rows * n * 8 / out["ms_multi_dot_k4"] / 1e6
        coef = torch.full((k, n), 1e-3, dtype=torch.complex128, device="cuda")
        out["ms_lincomb_k4"] = ev(lambda: mrhs.mrhs_blas_lincomb(basis[k], basis, k, coef, -1.0, rows, n,
                                                                  mrhs.MRHS_FP32))
        out["GBs_lincomb_k4"] = (k + 2) * rows * n * 8 / out["ms_lincomb_k4"] / 1e6
        return print(json.dumps(out), flush=True)
    if name == "coarse":
        return print(json.dumps(run_coarse_case(mrhs, torch, reps)), flush=True)
    if name == "coarsest":
        return print(json.dumps(run_coarsest_case(mrhs, torch, reps, ev)), flush=True)
    dims = (24, 24, 24, 24) if name in ("stencil", "schur", "stencil-sweep") else (16, 16, 16, 16)
    V = volume(dims)
    U = synth.gauge_exp(dims, WORKLOAD["eps"], WORKLOAD["gauge_seed"])
    lat = mrhs.mrhs_create_lattice(dims, -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat, U)
    mrhs.mrhs_build_clover(lat, WORKLOAD["mass"], WORKLOAD["csw"])
    out["dims"] = list(dims)
    if name == "stencil-sweep":
        # the fine operator alone (FP32) at every RHS count: algorithmic GB/s and fraction of the measured
        # HBM bandwidth, bytes per site 576 + 192 n (4 links, compact clover, one spinor in and out per RHS)
        peak, kind = read_peaks()
        out["peak_GBs"] = peak
        out["sweep"] = []
        for nn in (1, 2, 4, 8, 12, 16, 24, 32, 48, 64):
            a = torch.randn((V, 12, nn), dtype=torch.complex64, device="cuda")
            o = torch.empty_like(a)
            ms = ev(lambda: mrhs.mrhs_apply_D(lat, a, o, nn, mrhs.MRHS_FP32, stream))
            gbs = V * (576 + 192 * nn) / ms / 1e6
            out["sweep"].append({"nrhs": nn, "ms": ms, "alg_GBs": gbs, "frac": gbs / peak})
            del a, o
    elif name == "stencil":
        a = torch.randn((V, 12, n), dtype=torch.complex64, device="cuda")
        o = torch.empty_like(a)
        out["ms_apply_fp32"] = ev(lambda: mrhs.mrhs_apply_D(lat, a, o, n, mrhs.MRHS_FP32, stream))
        out["alg_GBs"] = V * (576 + 192 * n) / out["ms_apply_fp32"] / 1e6
    elif name == "schur":
        a = torch.randn((V // 2, 12, n), dtype=torch.complex64, device="cuda")
        o = torch.empty_like(a)
        out["ms_hop_eo"] = ev(lambda: mrhs.mrhs_apply_hop_eo(lat, 0, a, o, n, stream))
        out["ms_schur"] = ev(lambda: mrhs.mrhs_apply_schur(lat, a, o, n, stream))
        # per output site of D_hat (two launches): 8 links 576 B, C^-1 or C 288 B, neighbours and output
        # 192 n B, and the site's own spinor in the C - 1/4 H launch 96 n B: 1728 + 480 n
        out["schur_alg_GBs"] = (V // 2) * (1728 + 480 * n) / out["ms_schur"] / 1e6
    elif name == "intergrid":
        p = mrhs.mrhs_mg_default_params()
        p.n_levels = 2
        for mu in range(4):
            p.block[0][mu] = 4
        p.n_vec[0] = 32
        p.setup_sweeps = 0
        p.max_rhs = n
        p.coarse_m = p.smooth_m = p.inner_m = p.outer_m = 2
        p.coarse_precision = mrhs.MRHS_FP16
        p.use_graph = 0
        mg = mrhs.mrhs_setup_mg(lat, p)
        f = torch.randn((V, 12, n), dtype=torch.complex64, device="cuda")
        c = torch.randn((V // 256, 64, n), dtype=torch.complex64, device="cuda")
        out["ms_restrict_api"] = ev(lambda: mrhs.mrhs_restrict(mg, 0, f, c, n))
        out["ms_prolong"] = ev(lambda: mrhs.mrhs_prolong(mg, 0, c, f, n))
        mrhs.mrhs_destroy_mg(mg)
    else:
        raise SystemExit(f"unknown case {name}")
    mrhs.mrhs_destroy_lattice(lat)
    print(json.dumps(out), flush=True)


def run_batch_case(reps):
    """Uneven MRHS blocks (the serving mix: two resident volumes, requests of a few sources): the FP32 fine
    operator in its residual form on each block by separate launches, against one fused persistent
    launch (mrhs_apply_D_batch) over all of them.  Algorithmic bytes per block: V (576 + 192 n) + V 96 n (y)."""
    import torch

    import synth
    from paper_2211_13719_gb300 import build as _build
    from paper_2211_13719_gb300 import mrhs
    _build.build()
    mixes = {"serving-size": [((16, 16, 16, 32), 12), ((16, 16, 16, 32), 6), ((8, 8, 8, 16), 4),
                              ((12, 12, 12, 24), 8), ((16, 16, 16, 32), 2), ((8, 8, 8, 16), 12)],
             "small": [((8, 8, 8, 8), 4), ((8, 8, 8, 16), 2), ((4, 4, 4, 8), 8), ((8, 8, 8, 8), 12),
                       ((6, 6, 6, 6), 6), ((8, 8, 8, 8), 2), ((4, 4, 8, 8), 16), ((6, 6, 6, 6), 4)]}
    out = {"case": "batch", "mixes": []}
    for name, mix in mixes.items():
        out["mixes"].append(dict(name=name, **_batch_mix(mrhs, torch, synth, mix, reps)))
    print(json.dumps(out), flush=True)


def _batch_mix(mrhs, torch, synth, mix, reps):
    stream = torch.cuda.current_stream()
    lats, items, alg = {}, [], 0
    for dims, n in mix:
        if dims not in lats:
            lat = mrhs.mrhs_create_lattice(dims, -1, torch.cuda.current_device())
            mrhs.mrhs_load_gauge(lat, synth.gauge_exp(dims, WORKLOAD["eps"], 1402))
            mrhs.mrhs_build_clover(lat, WORKLOAD["mass"], WORKLOAD["csw"])
            lats[dims] = lat
        V = volume(dims)
        x = torch.randn((V, 12, n), dtype=torch.complex64, device="cuda")
        y = torch.randn_like(x)
        o = torch.empty_like(x)
        items.append((lats[dims], x, o, y, n))
        alg += V * (576 + 192 * n) + V * 96 * n

    def separate():
        for lat, x, o, y, n in items:
            mrhs.mrhs_residual_D(lat, x, y, o, n, mrhs.MRHS_FP32, stream)

    def fused():
        mrhs.mrhs_apply_D_batch(items, stream)

    def ev(fn):
        for _ in range(5):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_sep, ms_fused = ev(separate), ev(fused)
    out = {"blocks": [[list(d), n] for d, n in mix], "alg_bytes": alg,
           "ms_separate_launches": ms_sep, "ms_fused_launch": ms_fused, "speedup": ms_sep / ms_fused,
           "alg_GBs_separate": alg / ms_sep / 1e6, "alg_GBs_fused": alg / ms_fused / 1e6}
    for lat in lats.values():
        mrhs.mrhs_destroy_lattice(lat)
    return out


def run_c0_case(reps):
    """The small plain solve on the GPU: 8^4, antiperiodic t, U = exp(i 0.4 H) (seed 1001), m = -0.2, c_sw = 1,
    4 Gaussian sources, 2-level MG with 4^4 aggregates and 8 null vectors (nc = 16: the FP32 CUDA-core coarse
    stencil), outer FP64 FGMRES to 1e-10; seconds per 4-RHS solve after setup."""
    import numpy as np
    import torch

    import synth
    from paper_2211_13719_gb300 import build as _build
    from paper_2211_13719_gb300 import mrhs
    _build.build()
    dims, n = (8, 8, 8, 8), 4
    V = volume(dims)
    lat = mrhs.mrhs_create_lattice(dims, -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat, synth.gauge_exp(dims, 0.4, 1001))
    mrhs.mrhs_build_clover(lat, -0.2, 1.0)
    p = mrhs.mrhs_mg_default_params()
    p.n_levels = 2
    for mu in range(4):
        p.block[0][mu] = 4
    p.n_vec[0] = 8
    p.setup_sweeps = 4
    p.max_rhs = n
    p.coarse_precision = mrhs.MRHS_FP32
    p.coarse_m = 16
    p.coarse_cycles = 2
    p.smooth_m = 4
    p.smoother_evenodd = 0
    t0 = time.perf_counter()
    mg = mrhs.mrhs_setup_mg(lat, p)
    setup = time.perf_counter() - t0
    b = torch.from_numpy(synth.gaussian_field(V, 12, n, 2001)).cuda()
    x = torch.zeros_like(b)
    rel = np.zeros(n)
    times = []
    for i in range(reps + 1):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status, st = mrhs.mrhs_solve(mg, b, x, n, 1e-10, rel)
        torch.cuda.synchronize()
        if i:
            times.append(time.perf_counter() - t0)
    out = {"case": "c0", "setup_s": setup, "solve_4rhs_s": min(times), "outer_iters": st.outer_iters,
           "inner_iters": st.inner_iters, "max_rel_residual": float(rel.max())}
    mrhs.mrhs_destroy_mg(mg)
    mrhs.mrhs_destroy_lattice(lat)
    print(json.dumps(out), flush=True)


def run_serving_case(args):
    """The serving workload at several offered loads (--serve-loads, default 0.5, 0.8, 0.95 of the
    saturated 48-RHS solve rate measured first), --serve-requests requests each (default here 500)."""
    import numpy as np
    import torch

    from paper_2211_13719_gb300 import build as _build
    from paper_2211_13719_gb300 import mrhs
    _build.build()
    w = dict(WORKLOAD)
    n = w["nrhs"]
    V = volume(w["dims"])
    U = gauge_field(w)
    lat = mrhs.mrhs_create_lattice(w["dims"], -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat, U)
    mrhs.mrhs_build_clover(lat, w["mass"], w["csw"])
    del U
    mg = mrhs.mrhs_setup_mg(lat, make_params(mrhs, n, mrhs.MRHS_FP16, 1))
    b = torch.randn((V, 12, n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    rel = np.zeros(n)
    for _ in range(2):
        x.zero_()
        mrhs.mrhs_solve(mg, b, x, n, w["tol"], rel)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        x.zero_()
        mrhs.mrhs_solve(mg, b, x, n, w["tol"], rel)
    torch.cuda.synchronize()
    saturated = 2 * n / (time.perf_counter() - t0)
    del b, x
    out = {"case": "serving", "saturated_solves_per_s": saturated, "loads": []}
    nreq = args.serve_requests if args.serve_requests != 24 else 500
    with ClockSampler(torch.cuda.current_device()) as clk:
        for load in [float(v) for v in args.serve_loads.split(",")]:
            out["loads"].append(run_serving(mrhs, mg, w, saturated, args, torch, np, load=load, nreq=nreq))
            print(json.dumps(out["loads"][-1]), flush=True)
    out["clocks"] = clk.summary()
    mrhs.mrhs_destroy_mg(mg)
    mrhs.mrhs_destroy_lattice(lat)
    print(json.dumps(out), flush=True)


def run_coarsest_case(mrhs, torch, reps, ev):
    """The coarsest solve at the benchmark's coarsest size (3^3x8 sites, nc = 64, 48 RHS, GMRES(14)) on a
    small 2-level hierarchy (fine 12^3x32, 4^4 aggregates, 32 null vectors): the persistent kernel against
    the launch-per-operation path, CUDA events per solve."""
    import synth
    dims = (12, 12, 12, 32)
    w = WORKLOAD
    U = synth.gauge_exp(dims, w["eps"], w["gauge_seed"])
    lat = mrhs.mrhs_create_lattice(dims, -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat, U)
    mrhs.mrhs_build_clover(lat, w["mass"], w["csw"])
    out = {"case": "coarsest", "fine_dims": list(dims), "nrhs": 48, "coarse_m": MG_PARAMS["coarse_m"]}
    for fused in (1, 0):
        p = mrhs.mrhs_mg_default_params()
        p.n_levels = 2
        for mu in range(4):
            p.block[0][mu] = 4
        p.n_vec[0] = 32
        p.max_rhs = 48
        p.coarse_precision = mrhs.MRHS_FP16
        p.setup_sweeps = 2
        p.coarse_m = MG_PARAMS["coarse_m"]
        p.coarse_fused = fused
        mg = mrhs.mrhs_setup_mg(lat, p)
        d, dof = mrhs.mrhs_mg_level_info(mg, 1)
        cv = torch.randn((volume(d), dof, 48), dtype=torch.complex64, device="cuda")
        co = torch.zeros_like(cv)
        out["coarsest_dims"] = list(d)
        out["persistent_kernel" if fused else "launch_per_operation"] = {
            "ms_per_solve": ev(lambda: mrhs.mrhs_coarsest_solve(mg, cv, co, 48)),
            "info": list(mrhs.mrhs_coarsest_fused_info(mg))}
        mrhs.mrhs_destroy_mg(mg)
    mrhs.mrhs_destroy_lattice(lat)
    return out


def run_coarse_case(mrhs, torch, reps):
    """Coarse level and intergrid operators on 24^4 (Haar gauge) with 4^4 aggregates and 32 null
    vectors: the 6^4 coarse lattice with nc = 64.  Per nRHS in {12, 24, 48}: the coarse stencil with FP32
    links on CUDA cores and with FP16 / BF16 links on the tensor cores (the kernel alone and the whole
    apply including the input's scale and packing passes), restriction and prolongation, and the batched
    multi-dot over 4 coarse vectors.  Algorithmic bytes per coarse site: links 9 x 64 x 64 complex
    (294,912 B FP32, 147,456 B 16-bit) plus the input and output vectors 2 x 64 x n x 8 B; per fine site
    for the transfers: P (32 vectors x 12 complex, 3072 B FP32 / 1536 B 16-bit) and the fine vector 96 n B."""
    import numpy as np

    import synth
    peak, kind = read_peaks()
    dims, block, N = (24, 24, 24, 24), (4, 4, 4, 4), 32
    V = volume(dims)
    U = synth.gauge_haar(dims, 1201)
    lat = mrhs.mrhs_create_lattice(dims, -1, torch.cuda.current_device())
    mrhs.mrhs_load_gauge(lat, U)
    mrhs.mrhs_build_clover(lat, -0.2, 1.0)
    vecs = np.ascontiguousarray(synth.gaussian_field(V, 12, N, 3201))
    stream = torch.cuda.current_stream()
    out = {"case": "coarse", "dims": list(dims), "coarse_dims": [6, 6, 6, 6], "nc": 64, "peak_GBs": peak,
           "peak_source": kind, "rows": []}
    Vc = V // 256

    def ev(fn):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def kernel_ms(name, fn):
        mrhs.mrhs_kernel_timer_start(name)
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        ms, cnt, _ = mrhs.mrhs_kernel_timer_stop()
        return ms / max(cnt, 1)

    mgs = {}
    for prec in (mrhs.MRHS_FP16, mrhs.MRHS_BF16):
        p = mrhs.mrhs_mg_default_params()
        p.n_levels = 2
        for mu in range(4):
            p.block[0][mu] = block[mu]
        p.n_vec[0] = N
        p.setup_sweeps = 0
        p.max_rhs = 48
        p.coarse_precision = prec
        p.use_graph = 0
        p.init_vecs[0] = vecs.ctypes.data
        mgs[prec] = mrhs.mrhs_setup_mg(lat, p)
    names = {mrhs.MRHS_FP32: "fp32", mrhs.MRHS_FP16: "fp16", mrhs.MRHS_BF16: "bf16"}
    for n in (12, 24, 48):
        phi = torch.randn((Vc, 64, n), dtype=torch.complex64, device="cuda")
        o = torch.empty_like(phi)
        row = {"nrhs": n}
        vec_b = 2 * 64 * n * 8
        for prec in (mrhs.MRHS_FP32, mrhs.MRHS_FP16, mrhs.MRHS_BF16):
            mg = mgs[mrhs.MRHS_BF16 if prec == mrhs.MRHS_BF16 else mrhs.MRHS_FP16]
            fn = lambda: mrhs.mrhs_coarse_apply(mg, 1, phi, o, n, prec, stream)  # noqa: E731
            ms_apply = ev(fn)
            link_b = 294912 if prec == mrhs.MRHS_FP32 else 147456
            alg = Vc * (link_b + vec_b)
            k = "k_coarse_fp32" if prec == mrhs.MRHS_FP32 else "k_coarse_tc"
            ms_k = kernel_ms(k, fn)
            row[names[prec]] = {"ms_apply": ms_apply, "ms_kernel": ms_k, "kernel": k,
                                "alg_bytes": alg, "alg_GBs_kernel": alg / ms_k / 1e6,
                                "frac_kernel": alg / ms_k / 1e6 / peak, "alg_GBs_apply": alg / ms_apply / 1e6,
                                "tflops_kernel": Vc * 9 * 64 * 64 * n * 8 / ms_k / 1e9}
        f = torch.randn((V, 12, n), dtype=torch.complex64, device="cuda")
        mg = mgs[mrhs.MRHS_FP16]
        ms_r = ev(lambda: mrhs.mrhs_restrict(mg, 0, f, phi, n, stream))
        ms_p = ev(lambda: mrhs.mrhs_prolong(mg, 0, phi, f, n, stream))
        tb = V * (1536 + 96 * n) + Vc * 64 * n * 8
        row["restrict_tc"] = {"ms": ms_r, "alg_GBs": tb / ms_r / 1e6, "frac": tb / ms_r / 1e6 / peak}
        row["prolong_tc"] = {"ms": ms_p, "alg_GBs": tb / ms_p / 1e6, "frac": tb / ms_p / 1e6 / peak}
        basis = torch.randn((5, Vc * 64, n), dtype=torch.complex64, device="cuda")
        h = torch.empty((4, n), dtype=torch.complex128, device="cuda")
        ms_d = ev(lambda: mrhs.mrhs_blas_multi_dot(basis, 4, basis[4], Vc * 64, n, mrhs.MRHS_FP32, h, stream))
        row["multi_dot_k4"] = {"ms": ms_d, "alg_GBs": 5 * Vc * 64 * n * 8 / ms_d / 1e6}
        out["rows"].append(row)
        del phi, o, f, basis
    for mg in mgs.values():
        mrhs.mrhs_destroy_mg(mg)
    mrhs.mrhs_destroy_lattice(lat)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=0)
    ap.add_argument("--plain-solves", type=int, default=2)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95", help="offered loads of --case serving")
    ap.add_argument("--smoother", default="evenodd", choices=["evenodd", "sap", "gmres"],
                    help="fine post-smoother: GMRES on the even-odd Schur complement (default), SAP, or GMRES on D")
    ap.add_argument("--coarse-smoother", default="gmres", choices=["gmres", "evenodd"],
                    help="intermediate-level post-smoother: GMRES on the level operator (default) or on its "
                         "coarse even-odd Schur complement")
    ap.add_argument("--coarse-solver", default="gmres", choices=["gmres", "gcrodr"],
                    help="coarsest-level solver: GMRES(coarse_m) (default) or GCRO-DR(coarse_m, --coarse-recycle) "
                         "with its recycle space carried across V-cycles")
    ap.add_argument("--coarse-recycle", type=int, default=4)
    ap.add_argument("--coarse-fused", type=int, default=1, choices=[0, 1],
                    help="1 (default): the coarsest GMRES cycle as one persistent kernel; 0: one launch per "
                         "operation")
    ap.add_argument("--coarse-m", type=int, default=0, help="override the coarsest Krylov length")
    ap.add_argument("--sap-mr", type=int, default=4)
    ap.add_argument("--sap-cycles", type=int, default=1)
    ap.add_argument("--case", default=None, choices=["stencil", "stencil-sweep", "schur", "intergrid", "blas",
                                                     "coarse", "coarsest", "oracle-table", "serving", "c0",
                                                     "batch"],
                    help="run a small profiling case of one kernel family instead of the benchmark")
    ap.add_argument("--case-reps", type=int, default=3)
    ap.add_argument("--blas-rows", type=int, default=16 ** 4 * 12,
                    help="rows of the blas case (221184: the intermediate level, 3456 sites x 64 dof)")
    args = ap.parse_args()
    if args.case == "batch":
        run_batch_case(max(args.case_reps, 20))
        return
    if args.case == "c0":
        run_c0_case(args.case_reps)
        return
    if args.case == "serving":
        run_serving_case(args)
        return
    if args.case == "oracle-table":
        for th in sorted({1, os.cpu_count() or 1}):
            print(json.dumps(oracle_table(th)), flush=True)
        return
    if args.case:
        run_case(args.case, args.case_reps, args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
