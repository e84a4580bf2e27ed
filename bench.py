#!/usr/bin/env python
"""Benchmark of the batched adjoint fit of the nside-64 patch-configuration scan on B300.

One step = the whole hot path over one batch: cell building, the persistent fit of every
(configuration x realization) problem (SED tables, pixel assembly, GLS solves, likelihood,
adjoint gradient, L-BFGS), the W.d reconstruction with residual diagnostics, and the selection.

Workload: nside 64, |b| > 20 deg (32512 pixels), 1000 K-means patch configurations with
(K_bd, K_Td, K_bs) log-uniform in 1..500, 10 noise realizations shared by all configurations
(10000 problems); seeded synthetic LiteBIRD-like skies (see synth/).

  python bench.py [--gpus N --steps K --warmup W]      # CUDA path (one JSON line on rank 0)
  python bench.py --impl reference                     # FP64 CPU oracle on a bounded sample
Multi-GPU (torchrun): rank r fits its own 1000 configurations (seed 4 + r): weak scaling.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# seeded K-means labelings are deterministic: keep them between runs (git-ignored input cache)
os.environ.setdefault("CSX_KMEANS_CACHE", os.path.join(ROOT, ".cache", "kmeans"))

METRIC = "config fits/s & cluster-pixel L+grad L evals/s at nside64 vs plain form; % HBM peak"
SCAN = dict(nside=64, nconf=1000, kmax=500, nreal=10, b_cut_deg=20.0)
BYTES_PER_PIXEL_EVAL = 120 + 12 + 4   # 15 bands x Q,U float32 + 3 int32 labels + hit weight
# algorithmic bytes of one cell evaluation of the moment path: a cell's 120 unique second-moment
# entries (15 x 15 symmetric, float32) and its three int32 patch labels. The implementation keeps
# residual moments about a reference point instead (R 120 + C 45 + Q 6 floats: 696 B with labels),
# for precision; the roofline counts the algorithmic figure.
BYTES_PER_CELL_EVAL = 480 + 12
IMPL_BYTES_PER_CELL_EVAL = 4 * (120 + 45 + 6) + 12
FLOPS_PER_CELL_EVAL = 4600   # FP32 operations of one cell's chi2 + gradient (FMA = 2)
FLOPS_PER_PIXEL_EVAL = 1000  # FP32 operations of one pixel's chi2 + gradient (FMA = 2)
# DRAM bytes (read + write) per unit from ncu captures of the current kernels (None until the
# kernel has been captured since its last change): the persistent fit per cell evaluation, the
# streaming kernel per pixel evaluation (full-sky nside-64 case, 100 realizations).
TRAFFIC_FIT_PER_CELL_EVAL = None
TRAFFIC_STREAM_PER_PIXEL = {"L_and_grad": 133.4, "L": 132.9, "L_and_grad_unplanned": 130.3,
                            "L_unplanned": 130.1}
TRAFFIC_CAPTURE = {"fit": None,
                   "stream": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_spectral_tma, "
                             "full-sky nside 64, 40 realizations (profile_cases stream 40; 252 MB "
                             "of data, streamed, so traffic scales with the pixels), per pixel "
                             "evaluation"}


def fp32_peak_tflops(sm_mhz):
    """148 SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ----------------------------------------------------------------------------- inputs --------
def make_inputs(rank: int, nconf: int):
    import numpy as np
    from synth import workloads
    wl = workloads.scan(nside=SCAN["nside"], nconf=nconf, kmax=SCAN["kmax"], nreal=SCAN["nreal"],
                        b_cut_deg=SCAN["b_cut_deg"], seed=4 + rank)
    F = wl.sky.nfreq
    nb32 = np.zeros(16, np.float32)
    nb32[:F] = wl.sky.ninv_band.astype(np.float32)
    beta0 = np.concatenate([np.tile(wl.beta0(c), wl.nreal) for c in range(wl.nconf)]).astype(np.float32)
    return dict(wl=wl, d32=wl.data(), nb32=nb32, w32=wl.sky.w.astype(np.float32),
                fg32=wl.foreground_padded(), labels=np.ascontiguousarray(wl.labels, dtype=np.int32),
                K=np.ascontiguousarray(wl.K, dtype=np.int32), beta0=beta0)


# ----------------------------------------------------------------------------- clocks --------
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def mark(self):
        """Index of the next sample (to cut out the timed window)."""
        return len(self.rows)

    def summary(self, lo=0, hi=None):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows[lo:hi]:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle --------
def _oracle_job(args):
    import numpy as np
    from oracle import fit as ofit
    nu, d64, ninv64, lab, K, beta0, lower, upper = args
    t = time.time()
    x, L, info = ofit.fit(nu, d64, ninv64, lab, K, beta0, lower, upper, polish=False)
    return time.time() - t, int(info["nit"])


def _oracle_jobs(inp, nsample: int, step: int):
    """Problems of a bounded host sample: realization 0 of configurations whose P lies nearest the
    scan's 10th percentile (fits of ~10 s of one core each); step k takes the next nsample."""
    import numpy as np
    from synth import workloads
    wl = inp["wl"]
    P = wl.P
    pq = float(np.percentile(P, 10))
    order = np.argsort(np.abs(P - pq), kind="stable")
    pick = [order[(step * nsample + i) % len(order)] for i in range(nsample)]
    F = wl.sky.nfreq
    ninv64 = inp["w32"].astype(np.float64)[:, None] * inp["nb32"][:F].astype(np.float64)
    d64 = inp["d32"][0, :, :, :F].astype(np.float64)
    jobs = [(wl.sky.nu, d64, ninv64, wl.labels[c], wl.K[c], wl.beta0(c), workloads.LOWER,
             workloads.UPPER) for c in pick]
    return jobs, [int(P[c]) for c in pick], pq


def oracle_procs() -> int:
    """Oracle worker processes: half the host's cores, at most 8 (the numpy oracle is memory-bound:
    more processes mostly slow each other down)."""
    return max(1, min(len(os.sched_getaffinity(0)) // 2, 8))


def oracle_sample(inp, step: int = 0, pool=None):
    """Fit a bounded, seeded sample of problems with the FP64 oracle on the host cores (one
    process per core, BLAS single-threaded): about 10-30 s of wall time."""
    import multiprocessing as mp
    import numpy as np
    wl = inp["wl"]
    nsample = oracle_procs()
    jobs, Ps, pq = _oracle_jobs(inp, nsample, step)
    own = pool is None
    if own:
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")
        pool = mp.get_context("spawn").Pool(nsample)
    t0 = time.time()
    done = list(pool.imap_unordered(_oracle_job, jobs))
    wall = time.time() - t0
    if own:
        pool.close()
        pool.join()
    n = len(done)
    return {"value": n / wall, "unit": "fits/s", "cores": nsample, "kind": "oracle",
            "sample": "%d of %d problems: realization 0 of the configurations with P nearest the "
                      "scan's 10th percentile (%d; P %d..%d), nside 64, 32512 pixels, FP64 "
                      "numpy/scipy L-BFGS-B (no Newton polish), one process per core; smaller P than "
                      "the scan's median (%d), so the host rate is an upper bound for the full mix"
                      % (n, wl.nconf * wl.nreal, int(round(pq)), min(Ps), max(Ps),
                         int(np.median(wl.P))),
            "wall_s": wall,
            "single_fit_s_mean": float(np.mean([d[0] for d in done])),
            "oracle_iters_mean": float(np.mean([d[1] for d in done]))}


def oracle_spectra_sample(inp, nprob: int = 10):
    """The residual-spectra oracle (total, systematic and statistical pseudo-spectra to l = 150 on
    the scan's cut sky) on one configuration's `nprob` realizations (seeded normal maps: the cost
    does not depend on their values), in this process with numpy's BLAS threads."""
    import numpy as np
    from oracle import spectra as osp
    try:
        from threadpoolctl import threadpool_info
        threads = max([int(i.get("num_threads", 1)) for i in threadpool_info()] or [1])
    except Exception:
        threads = 1
    wl = inp["wl"]
    rng = np.random.default_rng(0)
    s_hat = rng.normal(size=(nprob, wl.npix, 2))
    s_true = rng.normal(size=(wl.npix, 2))
    r_sys = 0.1 * rng.normal(size=(nprob, wl.npix, 2))
    t0 = time.time()
    osp.residual_spectra(SCAN["nside"], wl.sky.pix, s_hat, s_true, r_sys, SPECTRA["lmax"])
    wall = time.time() - t0
    return {"value": nprob / wall, "unit": "problems/s", "cores": threads, "kind": "oracle",
            "sample": "%d problems' residual maps (tot, syst, stat), nside 64 cut sky, l <= 150, "
                      "FP64 direct sums over the pixels" % nprob, "wall_s": wall}


# ----------------------------------------------------------------------------- CUDA arm -------
def run_csx(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_08463_b300 import csx

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    inp = make_inputs(rank, args.nconf)
    cpu_base = oracle_sample(inp) if (rank == 0 and world == 1 and not args.no_cpu) else None
    if cpu_base is not None and not args.no_spectra:
        cpu_base["residual_spectra"] = oracle_spectra_sample(inp)

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = inp["wl"]
    nconf, nreal, npix = wl.nconf, wl.nreal, wl.npix
    nprob = nconf * nreal
    dev = torch.device("cuda", local)
    d = torch.from_numpy(inp["d32"]).to(dev)
    w = torch.from_numpy(inp["w32"]).to(dev)
    fg = torch.from_numpy(inp["fg32"]).to(dev)
    labels = torch.from_numpy(inp["labels"]).to(dev)
    beta0 = torch.from_numpy(inp["beta0"]).to(dev)
    K = inp["K"]
    model = csx.Model(wl.sky.nu)
    sky = csx.Sky(d, noise="separable", ninv_band=inp["nb32"], w=w)
    opts = dict(path=args.path, threads=args.threads)
    tuned = None
    if args.path == "auto" and args.threads == 0:
        # launch configuration of the fit picked by timing the candidates on a sample of the scan
        # (untimed; re-tuned every run rather than read from a cache made by another build)
        from paper_2604_08463_b300 import autotune
        opts, entry = autotune.tune_fit(csx, model, sky, labels, K, beta0)
        tuned = {"chosen": "%s/%d" % (opts["path"], opts["threads"]), "candidates_ms": entry["ms"],
                 "sample": "the whole scan, every problem capped at 10 iterations"}
    path = opts["path"] if opts["path"] != "auto" else "moment"  # auto: moment (separable noise)
    _, _, ncell_d = csx.build_cells(labels, K)
    ncell = ncell_d.cpu().numpy().astype(np.float64)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        res = csx.fit_batch(model, sky, labels, K, beta0, **opts)
        rec = csx.reconstruct(model, sky, labels, K, res["beta"], d_fg=fg, metrics=True)
        vt, best = csx.select(rec["metrics"], nconf, nreal)
        if dist:  # the path's one exchange: every rank's metric rows, then the global selection
            csx.gather_select(rec["metrics"], nreal)
        return res, rec, vt, best

    # the clock sampler starts before the warm-up: starting nvidia-smi stalls CUDA launches briefly
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fit_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    rec_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    evals = []
    host_s = {"fit": 0.0, "reconstruct": 0.0, "select": 0.0}
    mark0 = sampler.mark()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 flush (outside the step for k = 0, inside the stream order otherwise)
        if k == 0:
            e0.record(stream)
        fit_ev[k][0].record(stream)
        t = time.perf_counter()
        res = csx.fit_batch(model, sky, labels, K, beta0, **opts)
        host_s["fit"] += time.perf_counter() - t
        fit_ev[k][1].record(stream)
        rec_ev[k][0].record(stream)
        t = time.perf_counter()
        rec = csx.reconstruct(model, sky, labels, K, res["beta"], d_fg=fg, metrics=True)
        host_s["reconstruct"] += time.perf_counter() - t
        t = time.perf_counter()
        vt, best = csx.select(rec["metrics"], nconf, nreal)
        if dist:
            csx.gather_select(rec["metrics"], nreal)
        host_s["select"] += time.perf_counter() - t
        rec_ev[k][1].record(stream)
        evals.append(res["nevals"])
    e1.record(stream)
    torch.cuda.synchronize()
    bounds = [e0] + [a for a, _ in fit_ev[1:]] + [e1]
    breakdown = {"fit_ms": None, "reconstruct_select_ms": statistics.mean(
        a.elapsed_time(b) for a, b in rec_ev),
        "host_call_ms": {k: 1e3 * v / args.steps for k, v in host_s.items()},
        "step_ms": [bounds[i].elapsed_time(bounds[i + 1]) for i in range(args.steps)],
        "start_to_first_fit_ms": e0.elapsed_time(fit_ev[0][0])}
    mark1 = sampler.mark()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    fit_ms = statistics.mean(a.elapsed_time(b) for a, b in fit_ev)
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())

    status = res["status"].cpu().numpy()
    iters = res["iters"].cpu().numpy()
    nev = torch.stack(evals).to(torch.float64).mean(0).cpu().numpy()
    conf_of = np.repeat(np.arange(nconf), nreal)
    if path == "stream":
        unit_evals = float(nev.sum()) * npix
        alg_bytes = unit_evals * BYTES_PER_PIXEL_EVAL
        alg_flops = unit_evals * FLOPS_PER_PIXEL_EVAL
    else:
        unit_evals = float((nev * ncell[conf_of]).sum())
        alg_bytes = unit_evals * BYTES_PER_CELL_EVAL
        alg_flops = unit_evals * FLOPS_PER_CELL_EVAL
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (fit_ms * 1e-3) / 1e9
    sampler.stop()
    clocks = sampler.summary(mark0, mark1)
    fp32_peak = fp32_peak_tflops(clocks["sm_mhz"] or 2032.0)
    achieved_tf = alg_flops / (fit_ms * 1e-3) / 1e12
    # one untimed fit with the other evaluation path, for comparison
    torch.cuda.synchronize()
    other = "stream" if path == "moment" else "moment"
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    res_o = csx.fit_batch(model, sky, labels, K, beta0, path=other)
    c1.record(stream)
    torch.cuda.synchronize()
    other_fit = {"path": other, "fit_ms": c0.elapsed_time(c1),
                 "converged": int((res_o["status"].cpu().numpy() == 0).sum()),
                 "iters_mean": float(res_o["iters"].cpu().numpy().mean())}

    # AdaTopK (App. A) on the same problems, untimed comparison with the L-BFGS fit
    ada = None
    if rank == 0 and not args.no_adatopk:
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        res_a = csx.fit_batch(model, sky, labels, K, beta0, solver="adatopk", max_iter=5000)
        a1.record(stream)
        torch.cuda.synchronize()
        st_a = res_a["status"].cpu().numpy()
        offs, _ = csx.param_offsets(K, nreal)
        ptype = np.concatenate([np.concatenate([np.full(int(k[j]), j) for j in range(3)])
                                for k in K for _ in range(nreal)])
        tolv = np.array([1e-3, 1e-2, 1e-3])[ptype]
        dev_ = np.abs(res_a["beta"].cpu().numpy() - res["beta"].cpu().numpy()) / tolv
        dL = res_a["L"].cpu().numpy() - res["L"].cpu().numpy()
        ada = {"fit_ms": a0.elapsed_time(a1), "converged": int((st_a == 0).sum()),
               "max_iter": int((st_a == 1).sum()), "line_search": int((st_a == 3).sum()),
               "iters_mean": float(res_a["iters"].cpu().numpy().mean()),
               "evals_mean": float(res_a["nevals"].cpu().numpy().mean()),
               "beta_vs_lbfgs_over_tol": {"p50": float(np.median(dev_)),
                                          "p99": float(np.percentile(dev_, 99)),
                                          "frac_above_1": float((dev_ > 1).mean())},
               "L_minus_lbfgs": {"median": float(np.median(dL)), "max": float(dL.max()),
                                 "frac_lower": float((dL < 0).mean())}}

    def leg(enabled, fn, *a):
        """A side measurement; an error in one is recorded in its key, not raised."""
        if rank != 0 or not enabled:
            return None
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001
            torch.cuda.synchronize()
            return {"error": "%s: %s" % (type(e).__name__, e)}

    streaming = leg(not args.no_stream, streaming_rates, csx, hbm)
    fullsky = leg(not args.no_fullsky, fullsky_fit_rates, csx)
    pipeline = leg(not args.no_pipeline, pipeline_rates, csx)
    kmeans_gpu = leg(not args.no_kmeans, kmeans_rates, csx, inp)
    spectra = leg(not args.no_spectra, spectra_rates, csx, inp, model, sky, labels, fg, res["beta"])

    # end to end: pinned host inputs -> device, step, results -> host
    e2e = None
    if args.e2e_steps > 0:
        h_d = torch.from_numpy(inp["d32"]).pin_memory()
        h_w = torch.from_numpy(inp["w32"]).pin_memory()
        h_fg = torch.from_numpy(inp["fg32"]).pin_memory()
        h_lab = torch.from_numpy(inp["labels"]).pin_memory()
        h_b0 = torch.from_numpy(inp["beta0"]).pin_memory()
        out_b = torch.empty(beta0.shape, dtype=torch.float32).pin_memory()
        out_L = torch.empty(nprob, dtype=torch.float64).pin_memory()
        out_s = torch.empty(nprob, dtype=torch.int32).pin_memory()
        out_v = torch.empty(nconf, dtype=torch.float64).pin_memory()
        out_best = torch.empty(1, dtype=torch.int32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in (h_d, h_w, h_fg, h_lab, h_b0))
        d2h = sum(t.numel() * t.element_size() for t in (out_b, out_L, out_s, out_v, out_best))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.e2e_steps):
            flush.zero_()
            d.copy_(h_d, non_blocking=True)
            w.copy_(h_w, non_blocking=True)
            fg.copy_(h_fg, non_blocking=True)
            labels.copy_(h_lab, non_blocking=True)
            beta0.copy_(h_b0, non_blocking=True)
            r2, _, v2, b2 = step()
            out_b.copy_(r2["beta"], non_blocking=True)
            out_L.copy_(r2["L"], non_blocking=True)
            out_s.copy_(r2["status"], non_blocking=True)
            out_v.copy_(v2, non_blocking=True)
            out_best.copy_(b2, non_blocking=True)
        s1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = s0.elapsed_time(s1) / args.e2e_steps
        if dist:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * nprob / (e2e_ms * 1e-3), "unit": "fits/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms}

    plain = None
    if rank == 0 and not args.no_plain:
        plain = plain_form(csx, model, sky, labels, inp, fit_ms / max(1.0, float(iters.mean())),
                           float(iters.mean()), nprob / (ms * 1e-3))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # the library kernels one step launches: fit descriptors, queue order (up to 16384
    # configurations), cells (moment path) and the fit; reconstruction descriptors, tables and
    # reconstruction; the selection (and the global selection when N > 1)
    launches_per_step = (2 + (1 if nconf <= 16384 else 0) + (1 if path == "moment" else 0) + 3 + 1
                         + (1 if dist else 0))
    # DRAM traffic of one fit launch from the ncu capture (moment path only), scaled by units
    # the DRAM traffic per cell evaluation was captured with 128-thread CTAs
    traffic = (TRAFFIC_FIT_PER_CELL_EVAL * unit_evals
               if TRAFFIC_FIT_PER_CELL_EVAL and path == "moment" and opts["threads"] in (0, 128)
               else None)
    frac_mem, frac_alu = achieved / hbm, achieved_tf / fp32_peak
    if frac_alu >= frac_mem:
        roof = {"kernel": "k_fit (persistent fit)", "bound": "alu", "achieved": achieved_tf,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": frac_alu,
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x median SM clock %.0f MHz"
                               % (clocks["sm_mhz"] or 2032.0),
                "flops_per_unit": FLOPS_PER_CELL_EVAL if path == "moment" else FLOPS_PER_PIXEL_EVAL,
                "units": unit_evals, "traffic": traffic,
                "memory_side": {"achieved_gbs": achieved, "peak_gbs": hbm, "frac": frac_mem}}
    else:
        roof = {"kernel": "k_fit (persistent fit)", "bound": "hbm", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": frac_mem,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_unit": BYTES_PER_CELL_EVAL if path == "moment" else BYTES_PER_PIXEL_EVAL,
                "units": unit_evals, "traffic": traffic,
                "alu_side": {"achieved_tflops": achieved_tf, "peak_tflops": fp32_peak,
                             "frac": frac_alu}}
    roof["unit_kind"] = "cell evaluations" if path == "moment" else "pixel evaluations"
    roof["traffic_source"] = TRAFFIC_CAPTURE["fit"] if traffic else None
    roof["impl_bytes_per_unit"] = IMPL_BYTES_PER_CELL_EVAL if path == "moment" else None
    line = {
        "metric": METRIC,
        "value": world * nprob / (ms_max * 1e-3),
        "unit": "fits/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP32 pixel arithmetic, FP64 sums)",
        "data": "synthetic (seeded LiteBIRD-like skies, K-means patches)",
        "config": {"workload": wl.name, "nside": SCAN["nside"], "npix": npix, "nconf": nconf,
                   "nreal": nreal, "problems_per_gpu": nprob, "mean_P": float(wl.P.mean()),
                   "max_P": int(wl.P.max()), "fit_path": path,
                   "l2": "256 MiB buffer written before every timed step (L2 is 126 MB)",
                   "parallelism": "weak: each rank fits its own 1000 configurations",
                   "fit_launch": tuned or dict(path=args.path, threads=args.threads)},
        # pixel-equivalent rate: the moment path evaluates cells, not pixels; this counts each
        # likelihood evaluation as the pixels it stands for
        "cluster_pixel_equivalent_evals_per_s": float(nev.sum()) * npix / (fit_ms * 1e-3),
        "cell_evals_per_s": float((nev * ncell[conf_of]).sum()) / (fit_ms * 1e-3),
        "mean_cells": float(ncell.mean()),
        "fit_ms": fit_ms,
        "breakdown": dict(breakdown, fit_ms=fit_ms),
        "fit_stats": {"converged": int((status == 0).sum()), "max_iter": int((status == 1).sum()),
                      "line_search": int((status == 3).sum()), "nonphysical": int((status == 2).sum()),
                      "iters_mean": float(iters.mean()), "evals_mean": float(nev.mean())},
        "other_path_fit": other_fit,
        "streaming_kernel": streaming,
        "adatopk_fit": ada,
        "kmeans": kmeans_gpu,
        "residual_spectra": spectra,
        "fullsky_fit": fullsky,
        "pipeline": pipeline,
        "roofline": roof,
        "cpu_baseline": cpu_base,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "plain_form": plain,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


STREAM = dict(nside=64, K=(100, 20, 30), nreal=100)


def streaming_rates(csx, hbm, ncall=20):
    """The streaming likelihood (+ adjoint gradient) kernel on its own: one call evaluates L (and
    dL/dbeta) of 100 problems (the realizations) of the full-sky nside-64 configuration with
    K = (100, 20, 30) and hit-count (separable) noise, 49152 pixels each: 629 MB of data, more
    than L2, so every call streams it from HBM. Timed with CUDA events over `ncall` back-to-back
    calls; a call is the SED-table kernel, two memsets and the streaming kernel."""
    import numpy as np
    import torch
    from synth import workloads
    wl = workloads.fullsky(STREAM["nside"], STREAM["K"], nreal=STREAM["nreal"])
    dev = torch.device("cuda", torch.cuda.current_device())
    d = torch.from_numpy(wl.data()).to(dev)
    nb = np.zeros(16, np.float32)
    nb[:wl.sky.nfreq] = wl.sky.ninv_band
    w = torch.from_numpy(wl.sky.w.astype(np.float32)).to(dev)
    lab = torch.from_numpy(np.ascontiguousarray(wl.labels[0], dtype=np.int32)).to(dev)
    K = wl.K[0]
    beta = torch.from_numpy(np.tile(wl.beta0(0), (wl.nreal, 1)).astype(np.float32)).to(dev)
    model = csx.Model(wl.sky.nu)
    sky = csx.Sky(d, noise="separable", ninv_band=nb, w=w)
    stream = torch.cuda.current_stream()
    units = wl.nreal * wl.npix
    out = {"workload": "fullsky_nside%d K=%s R=%d separable noise"
                       % (STREAM["nside"], [int(k) for k in K], wl.nreal),
           "pixels_per_call": units, "bytes_per_pixel": BYTES_PER_PIXEL_EVAL,
           "timing": "CUDA events around %d calls (tables kernel + memsets + streaming kernel)"
                     % ncall}
    from paper_2604_08463_b300 import autotune
    # cell plan of the labels (label-only, built once; the beta-dependent per-cell scalars and band
    # vectors are formed inside every timed call)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = csx.SpectralPlan(lab, K)
    out["plan"] = {"cells": plan.ncell, "build_ms": (time.perf_counter() - t0) * 1e3,
                   "timing": "host clock around csx_spectral_plan_create (synchronises)"}

    def planned(grad):
        return lambda model, sky, lab, K, beta: plan.grad(model, sky, beta, want_grad=grad)

    legs = (("L_and_grad", planned(True), True, True), ("L", planned(False), False, True),
            ("L_and_grad_unplanned", csx.spectral_grad, True, False),
            ("L_unplanned", csx.spectral_like, False, False))
    for name, fn, grad, use_plan in legs:
        # tile schedule chosen by timing every built schedule on this call shape (left in force)
        sched, entry = autotune.tune_stream(csx, model, sky, lab, K, beta, grad=grad,
                                            plan=plan if use_plan else None)
        for _ in range(3):
            fn(model, sky, lab, K, beta)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ncall):
            fn(model, sky, lab, K, beta)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / ncall
        gbs = units * BYTES_PER_PIXEL_EVAL / (ms * 1e-3) / 1e9
        tkey = ("L_and_grad" if grad else "L") + ("" if use_plan else "_unplanned")
        out[name] = {"ms_per_call": ms, "cluster_pixel_evals_per_s": units / (ms * 1e-3),
                     "entry": "csx_spectral_grad_plan" if use_plan else
                              ("csx_spectral_grad" if grad else "csx_spectral_like"),
                     "schedule": {"chosen": "%d/%d" % sched, "candidates_ms": entry["ms"],
                                  "unit": "pixels per tile / pipeline stages"},
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": gbs / hbm,
                                  "traffic": (TRAFFIC_STREAM_PER_PIXEL[tkey] * units
                                              if TRAFFIC_STREAM_PER_PIXEL.get(tkey) else None),
                                  "traffic_source": TRAFFIC_CAPTURE["stream"]
                                  if TRAFFIC_STREAM_PER_PIXEL.get(tkey) else None}}
    csx.stream_schedule(0, 0)
    plan.close()
    del d, sky
    torch.cuda.empty_cache()
    return out


def kmeans_rates(csx, inp):
    """GPU spherical K-means (the step before the hot path): every distinct patch count of the
    scan (one labeling each, 32512 cut-sky pixels) in one launch, timed with CUDA events, and
    checked against the scan's labels from the input generator (bit-exact)."""
    import numpy as np
    import torch
    from synth import healpix, kmeans as km
    wl = inp["wl"]
    pix = healpix.galactic_cut(SCAN["nside"], SCAN["b_cut_deg"])
    vec = healpix.unit_vectors(SCAN["nside"])[pix]
    n = vec.shape[0]
    ks = sorted({int(k) for k in wl.K.reshape(-1)})
    init = [km.init_indices(n, k, 100 + k) for k in ks if 1 < k < n]
    vd = torch.from_numpy(vec).to(torch.device("cuda", torch.cuda.current_device()))
    csx.kmeans(vd, ks, init)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lab, iters = csx.kmeans(vd, ks, init)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lab = lab.cpu().numpy()
    # the generator's labeling of each K, from the scan's configurations
    ref = {}
    for c in range(wl.nconf):
        for j in range(3):
            ref.setdefault(int(wl.K[c, j]), wl.labels[c, j])
    mismatched = sum(int(not np.array_equal(lab[i], ref[k])) for i, k in enumerate(ks))
    # the host generator (the same Lloyd iterations in numpy, one process) on a bounded sample:
    # the labelings of the largest K, where the work per labeling is largest
    import time as _t
    big = [k for k in ks if 1 < k < n][-2:]
    h0 = _t.time()
    for k in big:
        km.spherical_kmeans(vec, k, 100 + k)
    host_s = _t.time() - h0
    return {"labelings": len(ks), "pixels": n, "ms": ms, "labelings_per_s": len(ks) / (ms * 1e-3),
            "host_generator": {"labelings": len(big), "K": big, "s": host_s,
                               "labelings_per_s": len(big) / host_s, "processes": 1},
            "iters_mean": float(iters.float().mean()), "mismatched_vs_generator": mismatched,
            "timing": "CUDA events around one csx_kmeans launch (one CTA per labeling)"}


PIPE = dict(nside=64, nconf=4000, kmax=1000, nreal=10, b_cut_deg=20.0, seed=4, chunk=250, lmax=150)


def pipeline_rates(csx):
    """The full pipeline at nside 64 with the |b| > 20 deg cut: 4000 patch configurations with
    (K_bd, K_Td, K_bs) log-uniform in 1..1000, 10 noise realizations each (the workload's 50
    realizations scaled to 10 to keep the bench within minutes; the cost per problem does not
    depend on R). Steps, each timed with CUDA events: GPU spherical K-means of every distinct K
    (bit-exact with the seeded host generator, whose ~900 labelings would take hours on the host;
    starting pixels drawn on the host), the batched adjoint fit of all 40000 problems, the
    reconstruction with the systematic and statistical residual metrics, the selection of the best
    configuration, and the residual spectra (l <= 150) of every configuration in chunks of 250."""
    import numpy as np
    import torch
    from synth import healpix, kmeans as km, sky as S, workloads
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    pix = healpix.galactic_cut(PIPE["nside"], PIPE["b_cut_deg"])
    sk = S.make_sky(PIPE["nside"], pix=pix, truth="smooth", hitcount=True)
    vec = healpix.unit_vectors(PIPE["nside"])[pix]
    n, nconf, nreal = vec.shape[0], PIPE["nconf"], PIPE["nreal"]
    kreq_all = workloads.sample_patch_counts(nconf, PIPE["kmax"], seed=PIPE["seed"])
    vd = torch.from_numpy(vec).to(dev)
    d = torch.from_numpy(sk.data_stack(nreal)).to(dev)
    nb = np.zeros(16, np.float32)
    nb[:sk.nfreq] = sk.ninv_band
    sky = csx.Sky(d, noise="separable", ninv_band=nb, w=torch.from_numpy(sk.w.astype(np.float32)).to(dev))
    model = csx.Model(sk.nu)
    fg = torch.from_numpy(sk.padded(sk.foreground)).to(dev)
    s_true = torch.tensor(np.asarray(sk.cmb, dtype=np.float32), device=dev)
    plan = csx.ShtPlan(PIPE["nside"], PIPE["lmax"], sk.pix)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def run(kreq):
        times = {}
        nc = kreq.shape[0]

        def timed(name, fn):
            a, b = ev(), ev()
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            times[name] = a.elapsed_time(b)
            return out

        ks = sorted({int(k) for k in kreq.ravel()})
        init = [km.init_indices(n, k, 100 + k) for k in ks if 1 < k < n]
        lab_k, _ = timed("kmeans_ms", lambda: csx.kmeans(vd, ks, init))
        pos = {k: i for i, k in enumerate(ks)}
        # per-configuration label array [C, 3, npix] from the labelings of the distinct K (input
        # assembly), and each labeling's patch count
        idx = torch.tensor([[pos[int(k)] for k in row] for row in kreq], device=dev)
        labels = lab_k[idx].contiguous()
        Keff = (lab_k.amax(dim=1) + 1).cpu().numpy()[idx.cpu().numpy()].astype(np.int32)
        P = Keff.sum(axis=1)
        beta0 = torch.tensor(np.concatenate([np.tile(np.concatenate(
            [np.full(int(Keff[c, j]), workloads.BETA0[j]) for j in range(3)]), nreal)
            for c in range(nc)]).astype(np.float32), device=dev)
        res = timed("fit_ms", lambda: csx.fit_batch(model, sky, labels, Keff, beta0))
        rec = timed("reconstruct_ms", lambda: csx.reconstruct(model, sky, labels, Keff, res["beta"],
                                                              d_fg=fg, metrics=True))
        vt, best = timed("select_ms", lambda: csx.select(rec["metrics"], nc, nreal))
        offs, _ = csx.param_offsets(Keff, nreal)
        offs = np.append(offs, int(P.sum()) * nreal)

        def spectra():
            out = []
            for c0 in range(0, nc, PIPE["chunk"]):
                c1 = min(nc, c0 + PIPE["chunk"])
                b = res["beta"][int(offs[c0 * nreal]):int(offs[c1 * nreal])]
                r = csx.reconstruct(model, sky, labels[c0:c1], Keff[c0:c1], b, d_fg=fg, s_hat=True,
                                    r_sys=True, metrics=False)
                out.append(csx.residual_spectra(plan, r["s_hat"], s_true, r["r_sys"], nreal)["stat"])
                del r
            return out
        timed("spectra_ms", spectra)
        return times, res, best, Keff, P, len(ks)

    run(kreq_all[:100])  # warm-up: scratch buffers grown, kernels loaded
    times, res, best, Keff, P, nks = run(kreq_all)
    ks = range(nks)
    total = sum(times.values())
    st = res["status"].cpu().numpy()
    return {"workload": "pipeline_nside64_b20_C%d_K%d_R%d" % (nconf, PIPE["kmax"], nreal),
            "configurations": nconf, "realizations": nreal, "problems": nconf * nreal,
            "mean_P": float(P.mean()), "max_P": int(P.max()), "distinct_K": len(ks),
            "stage_ms": times, "total_ms": total,
            "configurations_per_s": nconf / (total * 1e-3),
            "latency_per_configuration_ms": total / nconf,
            "fits_per_s": nconf * nreal / (times["fit_ms"] * 1e-3),
            "fit_stats": {"converged": int((st == 0).sum()), "max_iter": int((st == 1).sum()),
                          "line_search": int((st == 3).sum()),
                          "iters_mean": float(res["iters"].float().mean().item())},
            "best_configuration": int(best.item()), "K_best": Keff[int(best.item())].tolist(),
            "timing": "CUDA events around each stage, one pass after a warm-up pass on 100 "
                      "configurations; labels assembled from the distinct labelings on the device"}


FULLSKY = dict(nside=64, K=(100, 20, 30), nreal=100)


def fullsky_fit_rates(csx):
    """The full-sky nside-64 configuration with K = (100, 20, 30) and 100 noise realizations (hit-count
    noise, smooth truth): the batched adjoint fit of the 100 problems followed by the W d
    reconstruction of every realization (s_hat for all pixels, Q and U, three components), each
    timed with CUDA events."""
    import numpy as np
    import torch
    from synth import workloads
    wl = workloads.fullsky(FULLSKY["nside"], FULLSKY["K"], nreal=FULLSKY["nreal"])
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    d = torch.from_numpy(wl.data()).to(dev)
    nb = np.zeros(16, np.float32)
    nb[:wl.sky.nfreq] = wl.sky.ninv_band
    sky = csx.Sky(d, noise="separable", ninv_band=nb,
                  w=torch.from_numpy(wl.sky.w.astype(np.float32)).to(dev))
    model = csx.Model(wl.sky.nu)
    labels = torch.from_numpy(np.ascontiguousarray(wl.labels)).to(dev)
    beta0 = torch.tensor(np.tile(wl.beta0(0), wl.nreal).astype(np.float32), device=dev)
    out = {}
    for k in range(2):  # warm-up, then timed
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        res = csx.fit_batch(model, sky, labels, wl.K, beta0)
        e[1].record(stream)
        rec = csx.reconstruct(model, sky, labels, wl.K, res["beta"], s_hat=True, metrics=False)
        e[2].record(stream)
        torch.cuda.synchronize()
        out = {"fit_ms": e[0].elapsed_time(e[1]), "reconstruct_ms": e[1].elapsed_time(e[2])}
    st = res["status"].cpu().numpy()
    del rec, d, sky
    torch.cuda.empty_cache()
    return dict(out, workload="fullsky_nside64_K%s_R%d" % (list(FULLSKY["K"]), wl.nreal),
                fits_per_s=wl.nreal / (out["fit_ms"] * 1e-3),
                converged=int((st == 0).sum()),
                iters_mean=float(res["iters"].float().mean().item()))


SPECTRA = {"nconf": 100, "lmax": 150}
SM_MAX_MHZ = 2032.0


def spectra_rates(csx, inp, model, sky, labels, fg, beta, ncall=5):
    """Residual spectra (Sec. 2.5) of the first 100 configurations x their realizations at the
    step's fitted parameters: s_hat and r_sys from the reconstruction kernel (untimed), then the
    total, systematic and statistical (EE, BB) pseudo-spectra to l = 150 on the cut sky, each
    averaged over realizations, in one pass per call; CUDA events around `ncall` calls."""
    import numpy as np
    import torch
    wl = inp["wl"]
    nconf, nreal, lmax = min(SPECTRA["nconf"], wl.nconf), wl.nreal, SPECTRA["lmax"]
    K = inp["K"][:nconf]
    offs, _ = csx.param_offsets(inp["K"], nreal)
    nq = nconf * nreal
    b = beta[:int(offs[nq]) if nq < len(offs) else beta.numel()].contiguous()
    rec = csx.reconstruct(model, sky, labels[:nconf].contiguous(), K, b, d_fg=fg, s_hat=True,
                          r_sys=True, metrics=False)
    dev = beta.device
    s_true = torch.tensor(np.asarray(wl.sky.cmb, dtype=np.float32), device=dev)
    plan = csx.ShtPlan(SCAN["nside"], lmax, wl.sky.pix)
    out = csx.residual_spectra(plan, rec["s_hat"], s_true, rec["r_sys"], nreal)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ncall):
        out = csx.residual_spectra(plan, rec["s_hat"], s_true, rec["r_sys"], nreal)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / ncall
    nprob = nconf * nreal
    # algorithmic FP32 work: two transforms per problem (s_hat - s_true and r_sys; the statistical
    # residual's coefficients are their difference): ring sums 2 x (real x complex) per (pixel, m),
    # harmonic sums 4 x (real x complex) per (ring, l, m)
    from synth import healpix
    zc, _ = healpix.pixel_centres(SCAN["nside"])
    nring = np.unique(zc[np.asarray(wl.sky.pix)]).size
    nlm = sum(lmax - max(m, 2) + 1 for m in range(lmax + 1) if max(m, 2) <= lmax)
    flops = 2 * nprob * (8.0 * wl.npix * (lmax + 1) + 16.0 * nring * nlm)
    peak = fp32_peak_tflops(SM_MAX_MHZ)
    tf = flops / (ms * 1e-3) / 1e12
    bb = out["stat"][:, 1, 2:].cpu().numpy()
    del rec, out
    torch.cuda.empty_cache()
    return {"configurations": nconf, "realizations": nreal, "lmax": lmax, "problems_per_call": nprob,
            "transforms_per_call": 2 * nprob, "ms": ms, "problems_per_s": nprob / (ms * 1e-3),
            "stat_bb_mean_l2_150": float(bb.mean()),
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak,
                         "peak_source": "FP32 FMA lanes x SMs x 2 x max SM clock (148 x 128 x 2 x 2032 MHz)"},
            "timing": "CUDA events around %d residual_spectra calls (tot, syst, stat of every "
                      "configuration)" % ncall}


def plain_form(csx, model, sky, labels, inp, adj_ms_per_iter, adj_iters, adj_fits_per_s):
    """Plain GPU form: the same optimiser with central finite-difference gradients of the forward
    likelihood (2P+1 evaluations per gradient), on 20 configurations spanning the P range."""
    import numpy as np
    import torch
    wl = inp["wl"]
    P = wl.P
    qs = np.quantile(P, np.linspace(0.0, 1.0, 20))
    pick = sorted({int(np.argmin(np.abs(P - q))) for q in qs})
    sub_lab = labels[pick].contiguous()
    K = inp["K"][pick]
    b0 = torch.tensor(np.concatenate([np.tile(wl.beta0(c), wl.nreal) for c in pick]),
                      dtype=torch.float32, device=labels.device)
    max_iter = 10
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = csx.fit_batch(model, sky, sub_lab, K, b0, grad_mode="fd", path="stream", max_iter=max_iter)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = e0.elapsed_time(e1) * 1e-3  # device time of the launch (CUDA events)
    it = res["iters"].cpu().numpy()
    ne = res["nevals"].cpu().numpy()
    # time per quasi-Newton iteration of the plain form, scaled to the adjoint fit's iteration count
    nprob = len(pick) * wl.nreal
    per_iter = wall / max(1.0, float(it.mean()))
    extrap_fit_s = per_iter * adj_iters
    fits_per_s = nprob / extrap_fit_s
    return {"subset": "%d configurations (P quantiles %d..%d) x %d realizations, max_iter %d"
                      % (len(pick), int(P[pick].min()), int(P[pick].max()), wl.nreal, max_iter),
            "device_s": wall, "iters_mean": float(it.mean()), "evals_mean": float(ne.mean()),
            "fits_per_s_extrapolated": fits_per_s,
            "extrapolation": "subset device time per iteration x the adjoint fit's mean iterations "
                             "(%.1f); the subset's P mix differs from the full scan" % adj_iters,
            "adjoint_speedup": adj_fits_per_s / fits_per_s}


# ----------------------------------------------------------------------------- reference ------
def run_reference(args):
    """The oracle arm: each step fits a bounded sample of the scan's problems on the host cores
    (the worker pool is started during the warm-up, outside the timed steps)."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    inp = make_inputs(0, args.nconf)
    vals = []
    last = None
    with mp.get_context("spawn").Pool(oracle_procs()) as pool:
        pool.map(abs, range(64))  # warm-up: start the workers
        t0 = time.time()
        for k in range(args.steps):
            last = oracle_sample(inp, step=k, pool=pool)
            vals.append(last["value"])
        wall = time.time() - t0
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded LiteBIRD-like skies, K-means patches)",
            "config": {"workload": inp["wl"].name, "npix": inp["wl"].npix,
                       "note": "each step fits a bounded sample of the scan's problems on the host"},
            "cpu_baseline": dict(last, value=v),
            "e2e": {"value": v, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["csx", "reference"], default="csx")
    ap.add_argument("--path", choices=["auto", "stream", "moment"], default="auto")
    ap.add_argument("--nconf", type=int, default=SCAN["nconf"])
    ap.add_argument("--threads", type=int, default=0, help="fit CTA size (0 = automatic)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-stream", action="store_true", help="skip the streaming-kernel rates")
    ap.add_argument("--no-adatopk", action="store_true", help="skip the AdaTopK comparison fit")
    ap.add_argument("--no-kmeans", action="store_true", help="skip the GPU K-means rates")
    ap.add_argument("--no-spectra", action="store_true", help="skip the residual-spectra rates")
    ap.add_argument("--no-fullsky", action="store_true", help="skip the full-sky fit leg")
    ap.add_argument("--no-pipeline", action="store_true", help="skip the full-pipeline leg")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_csx(args)


if __name__ == "__main__":
    main()
