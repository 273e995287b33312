"""Benchmark of the sparse w-projection hot path on the paper-scale workload.

Workload (synthetic stand-in for the paper's M31/30Dor experiments): 256 x 256
sky of 200 Gaussian blobs, M = 32768 visibilities with radially Gaussian
(u, v) (sigma = 0.25 B, truncated to the band disk), w_d ~ U[0, 1], 2x padded
512^2 grid, KB W = 4, e = 0.99, exact chirp, complex64 G, 30 dB noise.

A step is one Douglas-Rachford iteration of the BPDN solve (10 dual
forward-backward iterations, each a Phi and a Phi^H, plus one Phi^H and the
prox update): 10.5 Phi+Phi^H pairs.  G is built once before the timed region
by the same library (the build is timed separately and reported as w-kernels
built per second).  Metric: Phi+Phi^H pairs per second, whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica (seed = rank); no collective on
the data path, timing is the max over ranks (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1307_3424_gb300 import synth  # noqa: E402

METRIC = "phi_phiH_pairs_per_s"
UNIT = "pairs/s"
INNER = 10
PAIRS_PER_STEP = INNER + 0.5          # 10 Phi + 11 Phi^H


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e", type=float, default=0.99)
    ap.add_argument("--value-dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--report-snr", action="store_true",
                    help="after the timed regions, continue the solve to the workload's DR iterations and "
                         "report the reconstruction SNR")
    ap.add_argument("--cpu-sample-rows", type=int, default=512,
                    help="rows of the oracle sample timed on the host cores (a few seconds of host work)")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "precision", "batched", "learned", "spread", "build", "gemm"])
    ap.add_argument("--spread-seeds", type=int, default=3, help="spread workload: simulations per point")
    ap.add_argument("--spread-iters", type=int, default=200, help="spread workload: DR iterations")
    ap.add_argument("--train-kernels", type=int, default=2 ** 20, help="learned workload: training kernels")
    ap.add_argument("--train-steps", type=int, default=1024, help="learned workload: Adam steps (batch 4096)")
    ap.add_argument("--batch-problems", type=int, default=None, help="problems of the batched workload")
    ap.add_argument("--no-plain", action="store_true", help="batched workload: skip the one-by-one comparison")
    ap.add_argument("--index-format", default="auto", choices=["auto", "columns", "mask", "runs"])
    ap.add_argument("--build-workload", default="paper", choices=["paper", "precision"],
                    help="build workload: the paper-scale case (or --n / --m) or the precision-form case")
    ap.add_argument("--n", type=int, default=None, help="image side of a smaller profiling case")
    ap.add_argument("--m", type=int, default=None, help="visibilities of a smaller profiling case")
    return ap.parse_args()


def workload(args):
    """The paper-scale workload, the precision-form workload (--workload
    precision: N=1024, M=2^21, S(w) boxes), or a smaller case of the paper-scale
    recipe (profiling)."""
    if args.workload == "precision":
        if args.m is None:
            return synth.PRECISION
        import dataclasses
        return dataclasses.replace(synth.PRECISION, name=f"{synth.PRECISION.name}_m{args.m}", M=args.m)
    wl = synth.PAPER_SCALE
    if args.n is None and args.m is None:
        return wl
    import dataclasses
    n = args.n or wl.N
    m = args.m or wl.M
    blobs = max(1, int(round(wl.n_blobs * (n / wl.N) ** 2)))
    return dataclasses.replace(wl, name=f"blobs{n}_m{m}", N=n, M=m, n_blobs=blobs)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_times_max(times_ms, ws, device=None):
    """Job time of weak-scaled replicas: the maximum over ranks of each timed
    region (a no-op for one process).  Collective over the default process
    group (NCCL on GPUs, gloo in the CPU tests)."""
    if ws <= 1:
        return [float(t) for t in times_ms]
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t) for t in times_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return [float(v) for v in tt.cpu()]


def job_rate(units_per_rank, ws, t_ms):
    """Whole-job throughput: every rank processed units_per_rank in the job time."""
    return units_per_rank * ws / (t_ms * 1e-3)


def workload_config(wl, e, extra=None):
    cfg = {"workload": f"{wl.name}_e{e}", "N": wl.N, "G": 2 * wl.N, "M": wl.M, "e": e,
           "uv": f"{wl.uv} sigma={wl.sigma_uv}B", "wd_max": wl.wd_max, "kb_support": wl.W,
           "box": 2 * wl.N if wl.box == "G" else "rule S(w)", "chirp": "exact", "dr_inner_iters": INNER,
           "pairs_per_step": PAIRS_PER_STEP}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f.read().splitlines() if ln.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------
# oracle timing on host cores (bounded sample); shared by cpu_baseline and --impl reference
# ---------------------------------------------------------------------------------


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_rows(job):
    """Worker of the oracle pool: the oracle's rows of G for a block of visibilities."""
    N, L, uvw, e = job
    from oracle import wproj_oracle as O
    return O.build_G(O.Geometry(N, L), uvw, e)


class OracleSample:
    """A bounded sample of the workload for the FP64 oracle on the host cores.

    R rows drawn at random are built by the oracle as it stands (`build_G`), in a
    pool of `cores` processes (spawned: the caller may hold a CUDA context).  One
    sample step is one Phi + Phi^H pair of the oracle restricted to those rows:
    the full-size FFT parts (Z A, F and their adjoints, numpy.fft, one thread)
    and the sparse products G_R X and G_R^H y over the R rows (scipy.sparse, the
    rows split into `cores` blocks run by as many threads; scipy releases the
    interpreter lock there).  A full pair over all M rows takes
    t_fft + t_sparse * M / R: that extrapolation is reported as such."""

    def __init__(self, wl, prob, e, n_rows, cores, seed=0):
        import concurrent.futures as cf
        import multiprocessing as mp
        from oracle import wproj_oracle as O
        self.O = O
        self.geo = O.Geometry(wl.N, prob.L)
        self.M = prob.uvw.shape[0]
        self.cores = max(1, int(cores))
        rng = np.random.default_rng(seed)
        self.rows = np.sort(rng.choice(self.M, min(n_rows, self.M), replace=False))
        jobs = [(wl.N, prob.L, np.ascontiguousarray(prob.uvw[r]), e)
                for r in np.array_split(self.rows, self.cores) if len(r)]
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            pool.map(_oracle_rows, [(wl.N, prob.L, prob.uvw[:1], e)] * len(jobs))   # start the workers
            t0 = time.perf_counter()
            self.blocks = pool.map(_oracle_rows, jobs)
            self.t_build = time.perf_counter() - t0
        self.nnz = int(sum(B.nnz for B in self.blocks))
        self.x = prob.x
        self.pool = cf.ThreadPoolExecutor(len(self.blocks))

    def step(self):
        """One sample pair; returns (t_fft, t_sparse) in seconds."""
        O, geo = self.O, self.geo
        t0 = time.perf_counter()
        X = O.F(geo, O.AZ(geo, self.x)).ravel()
        t1 = time.perf_counter()
        ys = list(self.pool.map(lambda B: B @ X, self.blocks))
        parts = list(self.pool.map(lambda a: a[0].T @ np.conj(a[1]), zip(self.blocks, ys)))
        Xt = np.conj(np.sum(parts, axis=0)).reshape(geo.G, geo.G)
        t2 = time.perf_counter()
        O.AZ_adj(geo, O.F_adj(geo, Xt))
        t3 = time.perf_counter()
        return (t1 - t0) + (t3 - t2), t2 - t1

    def full_pair_s(self, t_fft, t_sparse):
        return t_fft + t_sparse * self.M / len(self.rows)

    def describe(self):
        return (f"{len(self.rows)} of {self.M} rows ({self.nnz} entries) built by the FP64 oracle in "
                f"{self.t_build:.1f} s on {len(self.blocks)} processes "
                f"({len(self.rows) / self.t_build:.2f} w-kernels/s); a sample step = one Phi+Phi^H pair over "
                f"those rows: full-size numpy FFTs (1 thread) + scipy CSR products ({len(self.blocks)} threads); "
                f"value = full-workload pairs/s from t_fft + t_sparse * M/rows")

    def close(self):
        self.pool.shutdown()


def cpu_baseline(wl, prob, e, n_rows):
    t0 = time.perf_counter()
    smp = OracleSample(wl, prob, e, n_rows, host_cores())
    smp.step()
    best = min(smp.full_pair_s(*smp.step()) for _ in range(3))
    smp.close()
    return {"value": 1.0 / best, "unit": UNIT, "cores": len(smp.blocks), "kind": "oracle",
            "sample": smp.describe() + "; best of 3",
            "kernels_per_s": len(smp.rows) / smp.t_build,
            "wall_s": time.perf_counter() - t0}


# ---------------------------------------------------------------------------------
# reference arm: the oracle as the comparison program
# ---------------------------------------------------------------------------------


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload(args)
    prob = synth.make_problem(wl, seed=0)
    smp = OracleSample(wl, prob, args.e, args.cpu_sample_rows, host_cores())
    for _ in range(args.warmup):
        smp.step()
    steps = [smp.step() for _ in range(args.steps)]
    smp.close()
    timed_s = sum(a + b for a, b in steps)
    full_s = sum(smp.full_pair_s(a, b) for a, b in steps)
    value = args.steps / full_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": timed_s / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, args.e),
            "work_timed": {"step": "one Phi+Phi^H pair of the oracle over the row sample",
                           "rows_built": int(len(smp.rows)), "build_s": smp.t_build, "nnz_sample": smp.nnz,
                           "sample_pairs_timed": args.steps, "timed_s": timed_s},
            "extrapolation": {"value_is": "full-workload Phi+Phi^H pairs/s",
                              "per_step": "t_fft + t_sparse * M / rows", "M": int(smp.M),
                              "rows": int(len(smp.rows)), "full_pair_s_mean": full_s / args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(smp.blocks), "kind": "oracle",
                             "sample": smp.describe()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------


def read_profile_traffic(kernel: str, key: str = "traffic_bytes_per_launch"):
    """DRAM traffic of a kernel from a committed ncu summary in profiles/ (line
    '<key>: <n>' under '## <kernel>': per launch, or per entry of G)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(rf"##\s*{kernel}\b[^#]*?{key}:\s*([0-9.eE+]+)", txt, re.S)
    return float(m.group(1)) if m else None


def run_ours(args):
    import torch
    from paper_1307_3424_gb300 import wproj

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    wl = workload(args)
    e = args.e

    prob = synth.make_problem(wl, seed=rank)
    noise, sigma_n = synth.draw_noise(prob)
    plan = wproj.Plan(wl.N, prob.L, value_dtype=args.value_dtype, box=wl.box, index_format=args.index_format)
    uvw_d = torch.from_numpy(prob.uvw).to(dev)

    # build G (once untimed to load modules, then timed)
    plan.build_kernels(uvw_d, e)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.build_kernels(uvw_d, e)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    st = plan.stats()
    csrv = plan.csr()
    fmt, n_seg, stream_bytes = csrv.index_format, csrv.n_seg, csrv.stream_bytes
    del csrv
    nnz, M, G = st["nnz"], st["m"], plan.G

    # data and solver state
    x_d = torch.from_numpy(prob.x.astype(np.float32)).to(dev)
    y_d = plan.phi(x_d) + torch.from_numpy(noise.astype(np.complex64)).to(dev)
    eps = sigma_n * math.sqrt(M + 2 * math.sqrt(M))
    _, info = plan.solve_bpdn(y_d, eps, iters=1, inner_iters=INNER)      # power iteration + 1 iteration
    n2 = info.phi_norm2
    for _ in range(args.warmup):
        plan.solve_bpdn(y_d, eps, iters=1, inner_iters=INNER, phi_norm2=n2, resume=True, sync=False)
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    plan.set_timing(True)
    plan.reset_stats()
    x_out = torch.empty((wl.N, wl.N), dtype=torch.float32, device=dev)
    clocks = ClockSampler(dev.index if ws == 1 else local) if rank == 0 else None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()     # a profiler started with --profile-from-start off sees this region
    ev0.record(stream)
    for _ in range(args.steps):
        plan.solve_bpdn(y_d, eps, iters=1, inner_iters=INNER, phi_norm2=n2, resume=True, sync=False,
                        x_out=x_out)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop() if clocks else None
    t_ms = ev0.elapsed_time(ev1)
    kst = plan.stats()
    plan.set_timing(False)

    # ---- end to end through the public API with host buffers
    y_host = y_d.cpu().pin_memory()
    x_host = torch.empty((wl.N, wl.N), dtype=torch.float32).pin_memory()
    y_dev2 = torch.empty_like(y_d)
    plan.reset_stats()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        y_dev2.copy_(y_host, non_blocking=True)
        plan.solve_bpdn(y_dev2, eps, iters=1, inner_iters=INNER, phi_norm2=n2, resume=True, sync=False,
                        x_out=x_out)
        x_host.copy_(x_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e_ms = e0.elapsed_time(e1)

    t_ms, t_e2e_ms = reduce_times_max([t_ms, t_e2e_ms], ws, dev)

    # ---- reconstruction quality (outside the timed regions): the same solve
    # continued to the workload's Douglas-Rachford iterations
    snr = None
    if args.report_snr:
        done = 1 + args.warmup + 2 * args.steps
        rest = max(0, wl.dr_iters - done)
        if rest:
            plan.solve_bpdn(y_d, eps, iters=rest, inner_iters=INNER, phi_norm2=n2, resume=True, sync=False,
                            x_out=x_out)
        torch.cuda.synchronize()
        snr = {"dr_iters": max(done, wl.dr_iters),
               "snr_out_db": snr_out_db(prob.x, x_out.cpu().numpy().astype(np.float64))}

    # ---- roofline of the dominant kernel (degridding or gridding)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    b_val = 8 if args.value_dtype == "f32" else 4
    deg_ms = kst["t_degrid_ms"] / max(1, kst["n_degrid"])
    grid_ms = kst["t_grid_ms"] / max(1, kst["n_grid"])
    alg_deg = nnz * b_val + M * 8 + G * G * 8
    alg_grid = nnz * b_val + M * 8 + G * G * 8
    # G as each operator reads it: values + column indices, the tile-stream
    # records, or (run lengths) the row-major copy and the tile-major records
    if fmt == "columns":
        stored_deg = stored_grid = nnz * (b_val + 4)
    elif fmt == "runs":
        stored_deg, stored_grid = st["runs_bytes"], stream_bytes
    else:
        stored_deg = stored_grid = stream_bytes
    # kernel labels as in profiles/
    deg_name, grid_name = {"mask": ("k_stream_degrid", "k_stream_grid"), "runs": ("k_runs_degrid", "k_runs_grid"),
                           "columns": ("k_degrid", "k_grid_cells")}[fmt]
    if args.workload == "precision":   # the traffic figures in profiles/ are per workload
        deg_name += f"_precision_{args.value_dtype}"
        grid_name += f"_precision_{args.value_dtype}"
    if kst["t_degrid_ms"] >= kst["t_grid_ms"]:
        dom, ms, alg, kname, stored = "degrid", deg_ms, alg_deg, deg_name, stored_deg
    else:
        dom, ms, alg, kname, stored = "grid", grid_ms, alg_grid, grid_name, stored_grid
    achieved = alg / (ms * 1e-3) / 1e9
    roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": read_profile_traffic(kname),
            "peak_source": f"{peak_src} (copy bandwidth)",
            "algorithmic_bytes_per_launch": alg, "as_stored_bytes_per_launch": stored + M * 8 + G * G * 8,
            "as_stored_GBps": (stored + M * 8 + G * G * 8) / (ms * 1e-3) / 1e9,
            "ms_per_launch": ms,
            "degrid_ms": deg_ms, "grid_ms": grid_ms,
            "degrid_frac": alg_deg / (deg_ms * 1e-3) / 1e9 / hbm_peak,
            "grid_frac": alg_grid / (grid_ms * 1e-3) / 1e9 / hbm_peak,
            "degrid_as_stored_GBps": (stored_deg + M * 8 + G * G * 8) / (deg_ms * 1e-3) / 1e9,
            "grid_as_stored_GBps": (stored_grid + M * 8 + G * G * 8) / (grid_ms * 1e-3) / 1e9}

    value = job_rate(PAIRS_PER_STEP * args.steps, ws, t_ms)
    e2e_value = job_rate(PAIRS_PER_STEP * args.steps, ws, t_e2e_ms)
    out = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(wl, prob, e, args.cpu_sample_rows)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(wl, e, {"nnz": nnz, "segments": n_seg, "G_bytes": stored_deg + (
                                              stored_grid if fmt == "runs" else 0), "index_format": fmt,
                                              "value_dtype": args.value_dtype,
                                              "l2": "inputs larger than L2 (G exceeds L2 many times)",
                                              "parallelism": f"replicas x{ws}"}),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": M * 8,
                    "d2h_bytes_per_step": wl.N * wl.N * 4},
            "gpu_launches": None,
            "roofline": roof,
            "cpu_baseline": cpu,
            "build": {"ms": build_s * 1e3, "w_kernels_per_s": M / build_s, "nnz": nnz,
                      "nnz_per_row": nnz / M, "box": 2 * wl.N},
            "clocks": clk,
        }
        if snr is not None:
            line["reconstruction"] = snr
        out = line
    return out, kst


def run_batched(args):
    """The batched workload (256 problems, N in {64 .. 512}, M = f N^2): one step
    is one Douglas-Rachford iteration of every problem, replayed from the
    captured graph; the same problems run one by one through single plans are
    timed beside it (the plain GPU form)."""
    import torch
    from paper_1307_3424_gb300 import wproj

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    bw = synth.BATCHED
    probs = synth.make_batch(bw, seed=0, n_problems=args.batch_problems)
    ns = [p.wl.N for p in probs]
    ms = [p.uvw.shape[0] for p in probs]
    L = probs[0].L
    noise, sig = [], []
    for p in probs:
        nz, s_n = synth.draw_noise(p)
        noise.append(nz)
        sig.append(s_n)
    eps = [synth_eps(s_n, m) for s_n, m in zip(sig, ms)]
    uvw = torch.from_numpy(np.concatenate([p.uvw for p in probs])).to(dev)
    b = wproj.Batch(ns, L, box="rule")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.build_kernels(uvw, ms, bw.e)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sched = b.tune()
    info = b.info()
    x_cat = torch.from_numpy(np.concatenate([p.x.ravel() for p in probs]).astype(np.float32)).to(dev)
    y = b.phi(x_cat) + torch.from_numpy(np.concatenate(noise).astype(np.complex64)).to(dev)
    x_out = torch.empty(b.pixels, dtype=torch.float32, device=dev)
    b.solve_bpdn(y, eps, iters=1, inner_iters=INNER, x_out=x_out)       # power iterations, graph capture
    info = b.info()
    for _ in range(args.warmup):
        b.solve_bpdn(y, eps, iters=1, inner_iters=INNER, x_out=x_out, resume=True)
    torch.cuda.synchronize()
    l0 = b.info()["launches"]
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.solve_bpdn(y, eps, iters=1, inner_iters=INNER, x_out=x_out, resume=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    launches = b.info()["launches"] - l0
    snr_batch = [snr_out_db(p.x, xi.cpu().numpy().astype(np.float64)) for p, xi in zip(probs, b.split_images(x_out))]
    # end to end: visibilities from pinned host memory, images back, every step
    y_host = y.cpu().pin_memory()
    x_host = torch.empty(b.pixels, dtype=torch.float32).pin_memory()
    y2 = torch.empty_like(y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        y2.copy_(y_host, non_blocking=True)
        b.solve_bpdn(y2, eps, iters=1, inner_iters=INNER, x_out=x_out, resume=True)
        x_host.copy_(x_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1)

    plain = None
    if not args.no_plain:
        # the same problems one by one through single plans, same state
        plans = []
        for p, m_p, eps_p, y_p in zip(probs, ms, eps, b.split_vis(y)):
            pl = wproj.Plan(p.wl.N, L, box="rule", index_format="columns")
            pl.build_kernels(torch.from_numpy(p.uvw).to(dev), bw.e)
            y_p = y_p.contiguous()
            _, inf = pl.solve_bpdn(y_p, eps_p, iters=1 + args.warmup + args.steps, inner_iters=INNER)
            xo = torch.empty((p.wl.N, p.wl.N), dtype=torch.float32, device=dev)
            plans.append((pl, y_p, eps_p, inf.phi_norm2, xo))
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            for pl, y_p, eps_p, n2, xo in plans:
                pl.solve_bpdn(y_p, eps_p, iters=1, inner_iters=INNER, phi_norm2=n2, resume=True, sync=False,
                              x_out=xo)
        p1.record(stream)
        torch.cuda.synchronize()
        t_plain = p0.elapsed_time(p1)
        snr_plain = []
        for (pl, y_p, eps_p, n2, xo), p in zip(plans, probs):
            snr_plain.append(snr_out_db(p.x, xo.cpu().numpy().astype(np.float64)))
            pl.close()
        # both arms have now run 1 + warmup + 2 steps iterations (the batch: timed + e2e)
        plain = {"value": PAIRS_PER_STEP * args.steps / (t_plain * 1e-3), "unit": "batch pairs/s",
                 "ms_per_step": t_plain / args.steps, "form": "one plan per problem, solved one after another",
                 "speedup_of_batch": t_plain / t_ms}
        snr_b2 = [snr_out_db(p.x, xi.cpu().numpy().astype(np.float64)) for p, xi in zip(probs, b.split_images(x_out))]
        plain["max_abs_snr_diff_db"] = float(max(abs(a - c) for a, c in zip(snr_b2, snr_plain)))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    grid_cells = sum(4 * n * n for n in ns)
    alg = info["nnz"] * 8 + info["m"] * 8 + grid_cells * 8
    dom = "grid" if sched["grid_ms"] >= sched["degrid_ms"] else "degrid"
    ms_dom = max(sched["grid_ms"], sched["degrid_ms"])
    kname = "k_grid_cells_batch" if dom == "grid" else "k_degrid_batch"   # labels as in profiles/
    tr = read_profile_traffic(kname, "traffic_bytes_per_entry")   # from a smaller capture
    traffic = tr * info["nnz"] if tr is not None else None
    value = PAIRS_PER_STEP * args.steps / (t_ms * 1e-3)
    line = {
        "metric": "batch_phi_phiH_pairs_per_s", "value": value, "unit": "batch pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": bw.name, "problems": len(ns), "sides": {str(n): ns.count(n) for n in sorted(set(ns))},
                   "M_total": info["m"], "pixels_total": info["pixels"], "nnz": info["nnz"], "e": bw.e,
                   "w_c_max": f"U[0, {bw.wc_max}] per problem", "box": "rule S(w)", "dr_inner_iters": INNER,
                   "pairs_per_step": PAIRS_PER_STEP, "index_format": "columns",
                   "schedule": {"piece": sched["piece"], "chunk": sched["chunk"],
                                "lanes_per_piece": sched["lanes_per_piece"]},
                   "l2": "inputs larger than L2 (G exceeds L2 many times)", "parallelism": "one GPU"},
        "problem_pairs_per_s": value * len(ns),
        "e2e": {"value": PAIRS_PER_STEP * args.steps / (t_e2e * 1e-3), "unit": "batch pairs/s",
                "h2d_bytes_per_step": info["m"] * 8, "d2h_bytes_per_step": info["pixels"] * 4},
        "gpu_launches": int(launches),
        "launches_per_step": info["iter_launches"],
        "roofline": {"kernel": kname, "bound": "hbm",
                     "achieved": alg / (ms_dom * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": alg / (ms_dom * 1e-3) / 1e9 / hbm_peak, "traffic": traffic,
                     "traffic_source": "ncu DRAM bytes per entry of the 48-problem capture x nnz" if tr else None,
                     "peak_source": "measured (copy bandwidth)", "algorithmic_bytes_per_launch": alg,
                     "degrid_ms": sched["degrid_ms"], "grid_ms": sched["grid_ms"],
                     "timing": "autotuner's CUDA-event timing of the chosen schedules"},
        "plain_gpu": plain,
        "snr_db_mean": float(np.mean(snr_batch)),
        "build": {"ms": build_s * 1e3, "w_kernels_per_s": info["m"] / build_s, "nnz": info["nnz"]},
        "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def run_learned(args):
    """The learned-kernel form: the network trained on plain-build kernels (w_c ~
    U[0, 4], offsets U[0,1)^2) on the tensor cores, then the learned build of a
    2048^2 / M = 2^23 problem judged row by row against the plain build."""
    import torch
    from paper_1307_3424_gb300 import wproj

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    wl = synth.LEARNED
    if args.n or args.m:
        import dataclasses
        wl = dataclasses.replace(wl, N=args.n or wl.N, M=args.m or wl.M)
    L = synth.fov_L()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    flop_fwd = 2.0 * (3 * 256 + 2 * 256 * 256 + 256 * 3072)     # per kernel
    # ---- training data from the plain build
    m_t = args.train_kernels
    offs, wc = synth.mlp_samples(m_t, seed=0)
    uvw_t = torch.from_numpy(synth.mlp_uvw(offs, wc, wl.N, L, 1)).to(dev)
    pt = wproj.Plan(wl.N, L, box="rule", index_format="columns")
    pt.build_kernels(uvw_t, wl.e)
    x0, tv, tm = wproj.MLP.targets(pt, uvw_t)
    pt.close()
    net = wproj.MLP(torch.from_numpy(synth.mlp_init_params(0)))
    batch = 4096
    net.train(x0, tv, tm, batch=batch, steps=8, lr=1e-3)          # warm-up
    net.set_params(torch.from_numpy(synth.mlp_init_params(0)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(x0, tv, tm, batch=batch, steps=args.train_steps, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    train_tflops = args.train_steps * batch * 3.0 * flop_fwd / t_train / 1e12
    # ---- inference on the tensor cores (CUDA events)
    xi = x0[:65536].contiguous()
    net.forward(xi)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(5):
        net.forward(xi)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_inf = ev0.elapsed_time(ev1) / 5
    inf_tflops = 65536 * flop_fwd / (t_inf * 1e-3) / 1e12
    # the GEMM kernel alone on a compute-bound square product (8192^3, FP32 out)
    gs = 8192
    ga = torch.randn(gs, gs, device=dev).to(torch.bfloat16)
    gb = torch.randn(gs, gs, device=dev).to(torch.bfloat16)
    wproj.gemm_bf16(ga, gb)
    ev0.record(stream)
    for _ in range(5):
        wproj.gemm_bf16(ga, gb)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_sq = ev0.elapsed_time(ev1) / 5
    sq_tflops = 2.0 * gs ** 3 / (t_sq * 1e-3) / 1e12
    del ga, gb
    # held-out quality on the training distribution
    offs_h, wc_h = synth.mlp_samples(16384, seed=7)
    uvw_h = torch.from_numpy(synth.mlp_uvw(offs_h, wc_h, wl.N, L, 8)).to(dev)
    ph = wproj.Plan(wl.N, L, box="rule", index_format="columns")
    info_h, err_h = ph.build_kernels_learned(net, uvw_h, wl.e, rel_l2_max=1e-3)
    ph.close()
    eh = err_h.cpu().numpy()
    del x0, tv, tm
    # ---- deployment: plain build vs learned build with row-by-row fallback
    prob = synth.make_problem(wl, seed=0)
    uvw = torch.from_numpy(prob.uvw).to(dev)
    pd = wproj.Plan(wl.N, L, box="rule", index_format="columns")
    pd.build_kernels(uvw, wl.e)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pd.build_kernels(uvw, wl.e)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    info, err = pd.build_kernels_learned(net, uvw, wl.e, rel_l2_max=1e-3)
    e_np = err.cpu().numpy()
    pd.close()
    t_learned = (info["plain_ms"] + info["learned_ms"]) * 1e-3
    line = {
        "metric": "learned_w_kernels_per_s", "value": wl.M / t_learned, "unit": "w-kernels/s", "n_gpus": 1,
        "steps": args.train_steps, "warmup": 8, "ms_per_step": t_train / args.train_steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.N, "G": 2 * wl.N, "M": wl.M, "e": wl.e, "w_c": "U[0, 4]",
                   "box": "rule S(w)", "network": "3-256-256-256-3072 GELU, BF16 GEMMs (tcgen05), FP32 Adam",
                   "train_kernels": m_t, "train_batch": batch, "train_steps": args.train_steps,
                   "judge": "rel. L2 <= 1e-3 over the 32x32 window and predicted support >= e of the energy"},
        "plain_build_w_kernels_per_s": wl.M / t_plain,
        "learned": {"rows": info["rows"], "taken": info["learned"], "fraction": info["learned"] / info["rows"],
                    "rel_l2_mean": info["rel_l2_mean"], "rel_l2_median": float(np.median(e_np)),
                    "rel_l2_p10": float(np.percentile(e_np, 10)), "plain_ms": info["plain_ms"],
                    "infer_and_judge_ms": info["learned_ms"]},
        "held_out": {"rows": 16384, "rel_l2_median": float(np.median(eh)), "rel_l2_p10": float(np.percentile(eh, 10)),
                     "fraction_below_1e-2": float(np.mean(eh < 1e-2)), "fraction_below_1e-3": float(np.mean(eh < 1e-3))},
        "training": {"seconds": t_train, "samples_per_s": args.train_steps * batch / t_train,
                     "tflops": train_tflops, "loss_first": losses[0], "loss_last": float(np.mean(losses[-16:]))},
        "roofline": {"kernel": "k_gemm_ws (8192^3 BF16 product, FP32 out)", "bound": "tensor",
                     "achieved": sq_tflops, "peak": bf16_peak, "unit": "TFLOP/s", "frac": sq_tflops / bf16_peak,
                     "traffic": None, "peak_source": "measured (cuBLAS bf16 burst)", "ms": t_sq,
                     "mlp_forward": {"kernels": 65536, "ms": t_inf, "tflops": inf_tflops,
                                     "frac": inf_tflops / bf16_peak,
                                     "output_bytes": 65536 * 3072 * 4,
                                     "note": "bounded by writing the FP32 output of the last layer"}},
    }
    print(json.dumps(line))
    net.close()
    return 0


def run_spread(args):
    """The spread-spectrum experiment of Section 4 on blob skies, in paper mode
    (on-grid visibilities, Fourier-space upsampling, linear chirp, E = 0.75): the
    reconstruction SNR for w_d = 0, w_d ~ U[0, 1] and w_d = 1 against coverage,
    with the Dirac and the Daubechies-8 bases.  Each simulation draws its sky
    and cells once; the three w scenarios share them and the noise."""
    import torch
    from paper_1307_3424_gb300 import wproj

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    N, E, iters = args.n or 128, 0.75, args.spread_iters
    L = synth.fov_L()
    covs = [0.1, 0.2, 0.3, 0.5]
    scen = {"w0": 0.0, "varying": None, "max": 1.0}
    bases = {"dirac": 0, "db8": 8}
    snr = {b: {w: {c: [] for c in covs} for w in scen} for b in bases}
    t_iter = {b: [] for b in bases}
    plan = wproj.Plan(N, L, kb_support=1, chirp="linear", box="G", upsampling=True, index_format="columns")
    for seed in range(args.spread_seeds):
        for cov in covs:
            base = synth.paper_problem(N, cov, seed=seed)
            noise, sigma_n = synth.complex_noise(np.random.default_rng(1000 + seed), base.uvw.shape[0],
                                                 synth.noise_sigma(base.x, 30.0)), synth.noise_sigma(base.x, 30.0)
            eps = synth_eps(sigma_n, base.uvw.shape[0])
            xg = torch.from_numpy(base.x.astype(np.float32)).to(dev)
            for wname, wd in scen.items():
                prob = synth.paper_problem(N, cov, seed=seed, wd=wd)
                assert np.array_equal(prob.uvw[:, :2], base.uvw[:, :2])
                plan.build_kernels(torch.from_numpy(prob.uvw).to(dev), E)
                y = plan.phi(xg) + torch.from_numpy(noise.astype(np.complex64)).to(dev)
                for bname, psi in bases.items():
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    xr, _ = plan.solve_bpdn(y, eps, iters=iters, psi=psi, psi_levels=4, sync=False)
                    ev1.record(stream)
                    torch.cuda.synchronize()
                    t_iter[bname].append(ev0.elapsed_time(ev1) / iters)
                    snr[bname][wname][cov].append(snr_out_db(base.x, xr.cpu().numpy().astype(np.float64)))
    plan.close()
    # the wavelet transforms alone on an 8192^2 image (256 MB, larger than L2):
    # algorithmic bytes = one read and one write of every level's input
    nw, lev = 8192, 4
    xw = torch.randn(nw, nw, device=dev)
    aw = torch.empty_like(xw)
    wk = torch.empty(nw * nw // 2, device=dev)
    byt = sum(8.0 * (nw >> i) ** 2 for i in range(lev))
    wav = {}
    for name, fn, src, dst in (("dwt2", wproj.dwt2, xw, aw), ("idwt2", wproj.idwt2, aw, xw)):
        for _ in range(3):
            fn(src, lev, 8, out=dst)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(10):
            fn(src, lev, 8, out=dst)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / 10
        wav[name] = {"ms": ms, "gbs": byt / (ms * 1e-3) / 1e9}
    del xw, aw, wk
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    mean = {b: {w: {str(c): float(np.mean(v)) for c, v in snr[b][w].items()} for w in scen} for b in bases}
    sd = {b: {w: {str(c): float(np.std(v)) for c, v in snr[b][w].items()} for w in scen} for b in bases}
    lo = str(covs[0])
    db8 = mean["db8"]
    line = {
        "metric": "snr_out_db", "value": db8["varying"][lo], "unit": "dB", "n_gpus": 1,
        "steps": iters, "warmup": 0, "ms_per_step": float(np.median(t_iter["db8"])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"spread_paper{N}", "N": N, "G": 2 * N, "E": E, "coverages": covs,
                   "w_d": {"w0": 0, "varying": "U[0, 1]", "max": 1}, "sky": "20 Gaussian blobs",
                   "noise": "30 dB", "dr_iters": iters, "inner_iters": 10, "db8_levels": 4,
                   "simulations_per_point": args.spread_seeds},
        "snr_mean_db": mean, "snr_std_db": sd,
        "ms_per_dr_iteration": {b: float(np.median(v)) for b, v in t_iter.items()},
        "roofline": {"kernel": "k_dwt_level / k_idwt_level (Db8, 4 levels, 8192^2)", "bound": "hbm",
                     "achieved": wav["dwt2"]["gbs"], "peak": hbm, "unit": "GB/s", "frac": wav["dwt2"]["gbs"] / hbm,
                     "traffic": None, "idwt2_gbs": wav["idwt2"]["gbs"], "dwt2_ms": wav["dwt2"]["ms"],
                     "idwt2_ms": wav["idwt2"]["ms"], "peak_source": "measured (STREAM copy)"},
        "claims": {
            "db8_varying_beats_w0_at_10pc": db8["varying"][lo] > db8["w0"][lo],
            "db8_varying_minus_max_at_10pc_db": db8["varying"][lo] - db8["max"][lo],
            "dirac_spread_at_10pc_db": max(mean["dirac"][w][lo] for w in scen) - min(mean["dirac"][w][lo] for w in scen),
        },
    }
    print(json.dumps(line))
    return 0


def fp32_peak_tflops(peaks):
    """FP32 (non-tensor) arithmetic peak: 152 SMs x 128 FP32 lanes x 2 flop per
    FMA x the maximum SM clock."""
    return 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def run_build(args):
    """Part I alone (Sections 3.1-3.2): G of the paper-scale workload (or the
    --n / --m case, or --build-workload precision) built `steps` times after
    `warmup` builds.  Metric: w-kernels built per second over the wall time of
    the builds (a build sizes G exactly and synchronises); the library's
    CUDA-event timers give the device time of its stages (box tables + FFTs,
    selection + per-tile counts, emission)."""
    import torch
    from paper_1307_3424_gb300 import wproj

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = synth.PRECISION if args.build_workload == "precision" else workload(args)
    e = args.e if args.build_workload != "precision" else wl.e
    prob = synth.make_problem(wl, seed=0)
    plan = wproj.Plan(wl.N, prob.L, value_dtype=args.value_dtype, box=wl.box, index_format=args.index_format)
    uvw = torch.from_numpy(prob.uvw).to(dev)
    for _ in range(max(1, args.warmup)):
        plan.build_kernels(uvw, e)
    torch.cuda.synchronize()
    plan.set_timing(True)
    plan.reset_stats()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.build_kernels(uvw, e)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = plan.stats()
    plan.close()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    M = wl.M
    per = {k: st[f"t_build_{k}_ms"] / args.steps for k in ("fft", "select", "emit")}
    roof = None
    if wl.box == "G":
        S = 2 * wl.N
        fft_passes = st["n_build_fft"] / args.steps      # box batches transformed per build
        flop = 2 * M * 5.0 * S * S * math.log2(S * S)    # two passes over every box per build
        ach = flop / (per["fft"] * 1e-3) / 1e12
        pk = fp32_peak_tflops(peaks)
        roof = {"kernel": "k_box_rows + k_fft_cols (box tables and FFTs, both passes)", "bound": "alu",
                "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
                "flop_per_build": flop, "fft_ms_per_build": per["fft"], "batches_per_build": fft_passes}
    line = {
        "metric": "w_kernels_built_per_s", "value": M * args.steps / wall, "unit": "w-kernels/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl, e, {"nnz": st["nnz"], "box_min": st["box_min"], "box_max": st["box_max"],
                                          "value_dtype": args.value_dtype}),
        "stage_ms_per_build": per, "roofline": roof, "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def run_gemm(args):
    """The tensor-core GEMM alone (the MLP's contraction): C = A B^T for square
    BF16 matrices of side --n (default 8192), FP32 out, `steps` timed calls
    after `warmup`; FLOP rate against the measured BF16 peak."""
    import torch
    from paper_1307_3424_gb300 import wproj

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    n = args.n or 8192
    a = torch.randn(n, n, device=dev).to(torch.bfloat16)
    b = torch.randn(n, n, device=dev).to(torch.bfloat16)
    for _ in range(max(1, args.warmup)):
        wproj.gemm_bf16(a, b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    ev0.record(stream)
    for _ in range(args.steps):
        wproj.gemm_bf16(a, b)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    tflops = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    pk = float(peaks.get("bf16_tflops", 1900.0))
    line = {"metric": "gemm_bf16_tflops", "value": tflops, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"gemm{n}", "m": n, "n": n, "k": n, "out": "f32"},
            "roofline": {"kernel": "k_gemm_ws", "bound": "tensor", "achieved": tflops, "peak": pk,
                         "unit": "TFLOP/s", "frac": tflops / pk, "traffic": None,
                         "peak_source": "measured (cuBLAS bf16 burst)"},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def snr_out_db(x, x_rec):
    """SNR_out = 20 log10(std(x) / std(x - x_rec)) (Section 4.1)."""
    return 20.0 * math.log10(float(np.std(x)) / float(np.std(np.asarray(x) - np.asarray(x_rec))))


def synth_eps(sigma_n, M):
    """eps = sigma_n sqrt(M + 2 sqrt(M)), the chi^2 bound of the noise norm."""
    return sigma_n * math.sqrt(M + 2.0 * math.sqrt(M))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "spread":
        return run_spread(args)
    if args.workload == "build":
        return run_build(args)
    if args.workload == "gemm":
        return run_gemm(args)
    res = run_ours(args)
    out, kst = res
    if out is not None:
        out["gpu_launches"] = int(kst["launches"])
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
