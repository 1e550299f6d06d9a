#!/usr/bin/env python
"""Benchmark of the hot path: CG time-to-1e-10 and Dslash bandwidth at 32^3 x 64.

Workload (synthetic, seeded): a 32^3 x 64 SU(3) lattice with links
U = exp(iA), A traceless Hermitian with N(0, 0.25^2) entries (seed 2),
kappa = 0.156, antiperiodic time, a complex Gaussian source; M^dag M x = phi
is solved from x0 = 0 to an FP64 true relative residual of 1e-10.

One step = one mixed-precision solve (inner precision --inner, default FP16
storage with 12-real links and per-site FP32 norms, FP32 arithmetic, FP64
reliable updates every 50 iterations).  Printed as one JSON line:
  value         solves per second over all ranks (device-timed, data resident)
  e2e           the same through the C interface with pinned host buffers
                (gauge field and source copied in, solution copied out, every step)
  roofline      CG pass 2 of the inner precision (the largest kernel of the
                solve), timed with CUDA events on the library's stream, against
                the measured HBM copy bandwidth
  fp64          the plain FP64 CG on the same source (the comparison of the metric)
  cpu_baseline  the FP64 CPU oracle on a bounded sample, scaled to solves/s

--impl reference times the oracle instead (the CPU program of this project
written from the paper), on a bounded sample per step.
Multi-GPU runs (torchrun) are independent replicas: every rank solves its
own lattice; the time is the maximum over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG time-to-1e-10 & Dslash GB/s vs HBM peak at 32^3x64, mixed vs FP64"
DIMS = (32, 32, 32, 64)
SIGMA, SEED, KAPPA, TOL, RELIABLE = 0.25, 2, 0.156, 1e-10, 50
WORKLOAD = "cg_32x32x32x64"

# Algorithmic (DRAM-minimal) bytes per site, every link and spinor moved once.
GAUGE_B = {"f64": 576, "f32": 288, "f32_12": 192, "f16_12": 96, "bf16_12": 96, "df64": 576, "i16_12": 96}
SPINOR_B = {"f64": 192, "f32": 96, "f32_12": 96, "f16_12": 52, "bf16_12": 52, "df64": 192,
            "i16_12": 52}   # 16-bit: 48 + 4-byte norm
# one application of M: gauge + input spinor + output spinor
DSLASH_BYTES = {k: GAUGE_B[k] + 2 * SPINOR_B[k] for k in GAUGE_B}
# the three passes of a CG iteration:
#   k1  t = M p, |t|^2                          gauge + p + t
#   k2  r -= alpha M^dag t, x += alpha p, |r|^2  gauge + t + r (read, write) + x (read, write) + p
#   k3  p = r + beta p                          r + p (read, write)
# the low-precision solution x is stored in FP32 when the iteration vectors are 16-bit
X_B = {k: (96 if SPINOR_B[k] == 52 else SPINOR_B[k]) for k in SPINOR_B}
CG_BYTES = {k: {"k1": GAUGE_B[k] + 2 * SPINOR_B[k], "k2": GAUGE_B[k] + 4 * SPINOR_B[k] + 2 * X_B[k],
                "k3": 3 * SPINOR_B[k]} for k in GAUGE_B}
DSLASH_FLOPS = 1368
# DRAM traffic per site of the plain Dslash from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over sites), valid for the kernel sources with this
# hash; see profiles/.  Null when the kernel changed since the capture.
NCU_TRAFFIC = {
    # profiles/cg_pass2_f16_12_32x32x32x32.md
    "f16_12": {"bytes_per_site": 466.8, "src": "87e450e4b735615e"},
    # profiles/cg_pass2_i16_12_32x32x32x32.md
    "i16_12": {"bytes_per_site": 464.9, "src": "87e450e4b735615e"},
    # profiles/cg_pass2_f32_12_32x32x32x32.md
    "f32_12": {"bytes_per_site": 755.4, "src": "87e450e4b735615e"},
}


def kernel_source_hash():
    """Hash of the code (comments and blank space removed) of the files that define the
    CG passes, so that a comment edit does not void the traffic figures."""
    import re
    h = hashlib.sha256()
    for f in ("lq_device.cuh", "lq_dslash.cuh", "lq_internal.h", "k_cglo.cu"):
        text = open(os.path.join(ROOT, "paper_1207_2223_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        text = open(self.f.name).read()
        os.unlink(self.f.name)
        return self.summarise(text)

    @staticmethod
    def summarise(text):
        """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi's CSV."""
        rows = [ln.split(",") for ln in text.splitlines() if ln.strip()]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 8 for i in range(4) if r[5 + i].strip() == "Active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def make_inputs():
    from synth import Lattice, gauge_exp_iA, source
    lat = Lattice(DIMS)
    return lat, gauge_exp_iA(lat, SIGMA, SEED), source(lat, SEED)


def oracle_cg_iteration_seconds(U, phi, site_fraction=1):
    """Time the oracle's work for one CG iteration (M^dag M plus the vector updates).

    With site_fraction f > 1, M and M^dag are evaluated on a 1/f sample of the
    sites (same operator code, gathered) and the time is scaled by f."""
    import numpy as np
    from oracle.conventions import neighbours
    from oracle.wilson import apply_M
    nbr = neighbours(DIMS, True)
    V = U.shape[0]
    sites = None if site_fraction == 1 else np.arange(0, V, site_fraction)
    t0 = time.perf_counter()
    a = apply_M(U, phi, DIMS, KAPPA, True, False, sites, nbr)
    b = apply_M(U, phi, DIMS, KAPPA, True, True, sites, nbr)
    t1 = time.perf_counter()
    x = phi.copy()
    r = phi.copy()
    alpha = 0.5
    x = x + alpha * phi
    r = r - alpha * phi
    rr = np.vdot(r, r).real
    p = r + (rr / (rr + 1.0)) * phi
    t2 = time.perf_counter()
    del a, b, x, r, p
    return (t1 - t0) * site_fraction + (t2 - t1)


def measure_extras(lq, torch, dev):
    """Numbers beside the headline, each measured once outside the timed region:
    HMC trajectories at 16^4, the batched solve at 24^4 x 12, and CG time against
    iteration count with and without CUDA graphs (per-call overhead = intercept)."""
    import numpy as np
    from synth import Lattice, gauge_exp_iA, source, momenta, chi_noise, metropolis_uniform
    out = {}
    # HMC trajectories (beta 5.6, kappa 0.155, 20 leapfrog steps, tau 1, reunitarised exp(iA)
    # start, sigma 0.3) with the per-routine device-time split, 8^4 to 24^4; FP64 and mixed
    # solves at 16^4
    for dims in ((8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 24)):
        lat = Lattice(dims)
        U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 1, reunitarise=True)).to(dev)
        p0 = torch.from_numpy(momenta(lat, 1)).to(dev)
        chi = torch.from_numpy(chi_noise(lat, 1)).to(dev)
        u = metropolis_uniform(1)
        hmc = {}
        runs = (("f64", lq.LQ_F64), ("mixed_f16_12", lq.LQ_F16_12)) if dims[0] == 16 else (("mixed_f16_12", lq.LQ_F16_12),)
        for name, prec in runs:
            ctx = lq.lq_create(dims, True, torch.cuda.current_stream(dev).cuda_stream)
            try:
                lq.lq_gauge_set(ctx, U)
                r = lq.lq_hmc_trajectory(ctx, p0.clone(), chi, u, 5.6, 0.155, 20, 1.0, 1e-10, 20000, prec, 50)
            finally:
                lq.lq_destroy(ctx)
            dev_total = r["seconds_solve"] + r["seconds_gauge_force"] + r["seconds_fermion_force"] + \
                r["seconds_link_update"]
            hmc[name] = {"seconds": r["seconds"], "trajectories_per_s": 1.0 / r["seconds"], "dH": r["dH"],
                         "accepted": r["accepted"], "solves": r["solves"], "cg_iterations": r["cg_iterations"],
                         "plaquette": r["plaquette"],
                         "share": {"solve": r["seconds_solve"] / dev_total,
                                   "gauge_force": r["seconds_gauge_force"] / dev_total,
                                   "fermion_force": r["seconds_fermion_force"] / dev_total,
                                   "link_update": r["seconds_link_update"] / dev_total}}
        out["hmc_%dx%dx%dx%d" % dims] = hmc
    # batched solve: 24^4, kappa 0.155, seed 3, 12 right-hand sides sharing one gauge field
    dims = (24, 24, 24, 24)
    lat = Lattice(dims)
    U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 3)).to(dev)
    phis = torch.from_numpy(np.stack([source(lat, 3, i) for i in range(12)])).to(dev)
    ctx = lq.lq_create(dims, True, torch.cuda.current_stream(dev).cuda_stream)
    try:
        lq.lq_gauge_set(ctx, U)
        x = torch.zeros_like(phis)
        lq.lq_solve_batch([ctx], [x], [phis], [0.155], 12, 1e-10, 20000, lq.LQ_F16_12, 50)   # autotune
        t0 = time.perf_counter()
        status, st, iters, resid, _ = lq.lq_solve_batch([ctx], [x], [phis], [0.155], 12, 1e-10, 20000,
                                                        lq.LQ_F16_12, 50)
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        for i in range(12):
            xs = torch.zeros_like(phis[i])
            lq.lq_solve_MdagM(ctx, xs, phis[i], 0.155, 1e-10, 20000, lq.LQ_F16_12, 50)
        ts = time.perf_counter() - t0
    finally:
        lq.lq_destroy(ctx)
    out["batch_24x24x24x24_12rhs"] = {"seconds": tb, "sequential_seconds": ts, "iterations": st["iterations"],
                                      "max_true_rel_resid": float(resid.max())}
    # register ablation (paper Sec. 3-4): naive global-memory FP64 operator against the
    # optimised FP64 and FP32-12 ones, 32^3 x 64
    lat = Lattice(DIMS)
    U = torch.from_numpy(gauge_exp_iA(lat, SIGMA, SEED)).to(dev)
    phi = torch.from_numpy(source(lat, SEED)).to(dev)
    ctx = lq.lq_create(DIMS, True, torch.cuda.current_stream(dev).cuda_stream)
    try:
        lq.lq_gauge_set(ctx, U)
        out_t = torch.empty_like(phi)
        naive = lq.lq_apply_M_naive(ctx, out_t, phi, KAPPA, False, 3)
        opt64 = lq.lq_time_dslash(ctx, phi, KAPPA, False, lq.LQ_F64, 10, False)
        opt32 = lq.lq_time_dslash(ctx, phi, KAPPA, False, lq.LQ_F32_12, 20, False)
        del out_t
        # the force half: naive against optimised fermion-force kernel (X = the source)
        F = torch.empty((lat.V, 4, 8), dtype=torch.float64, device=dev)
        naive_f = lq.lq_fermion_force_naive(ctx, F, phi, KAPPA, 3)
        del F
        opt_f = lq.lq_time_fermion_force(ctx, phi, KAPPA, 10)
    finally:
        lq.lq_destroy(ctx)
    out["register_ablation_32x32x32x64"] = {"naive_f64_ms": naive, "optimised_f64_ms": opt64,
                                            "optimised_f32_12_ms": opt32, "f64_speedup": naive / opt64,
                                            "f32_12_speedup": naive / opt32,
                                            "naive_fermion_force_ms": naive_f, "optimised_fermion_force_ms": opt_f,
                                            "fermion_force_speedup": naive_f / opt_f}
    # CG time against iteration count, FP64 CG stopped by the iteration limit (tol 1e-30),
    # with and without CUDA graphs; 8^4 (launch-bound) and 16^4
    for dims in ((8, 8, 8, 8), (16, 16, 16, 16)):
        lat = Lattice(dims)
        U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 1)).to(dev)
        phi = torch.from_numpy(source(lat, 1)).to(dev)
        scan = {}
        for graphs in (1, 0):
            ctx = lq.lq_create(dims, True, torch.cuda.current_stream(dev).cuda_stream)
            try:
                lq.lq_gauge_set(ctx, U)
                lq.lq_set_option(ctx, lq.LQ_OPT_CUDA_GRAPHS, graphs)
                pts = []
                for n in (16, 64, 128, 256, 16, 64, 128, 256):
                    x = torch.zeros_like(phi)
                    t0 = time.perf_counter()
                    lq.lq_solve_MdagM(ctx, x, phi, 0.155, 1e-30, n, lq.LQ_F64, 0)
                    pts.append((n, time.perf_counter() - t0))
                pts = pts[4:]
                ns = np.array([q[0] for q in pts], dtype=float)
                ts = np.array([q[1] for q in pts])
                slope, icpt = np.polyfit(ns, ts, 1)
            finally:
                lq.lq_destroy(ctx)
            scan["graphs" if graphs else "no_graphs"] = {"seconds_per_iteration": slope, "intercept_s": icpt,
                                                         "points": [[int(a), b] for a, b in pts]}
        out["cg_time_vs_iterations_%dx%dx%dx%d" % dims] = scan
    return out


def run_hmc_ensemble(args):
    """A run of HMC trajectories (no timing contract).  Default: 32^4, beta 5.7, kappa 0.155,
    25 leapfrog steps, tau 1, mixed-precision solves, from the exp(iA) start (sigma 0.3, seed 8).
    --dims / --beta / --hmc-kappa / --md-steps / --trajectories / --start ordered select other
    runs (the paper's volume-scaling runs are 200 trajectories from an ordered start).  Prints
    one line per trajectory and a summary: acceptance, <exp(-Delta H)> and the plaquette over
    the second half of the run (after thermalisation), time per trajectory and its split."""
    import numpy as np
    import torch
    import paper_1207_2223_gb300 as lq
    from synth import Lattice, gauge_exp_iA, identity_gauge, momenta, chi_noise, metropolis_uniform
    dims = tuple(args.dims) if tuple(args.dims) != DIMS else (32, 32, 32, 32)
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    U0 = identity_gauge(lat) if args.start == "ordered" else gauge_exp_iA(lat, 0.3, 8)
    lq.lq_gauge_set(ctx, torch.from_numpy(U0).cuda())
    rows = []
    t0 = time.perf_counter()
    for traj in range(args.trajectories):
        p = torch.from_numpy(momenta(lat, 8, traj)).cuda()
        chi = torch.from_numpy(chi_noise(lat, 8, traj)).cuda()
        r = lq.lq_hmc_trajectory(ctx, p, chi, metropolis_uniform(8, traj), args.beta, args.hmc_kappa,
                                 args.md_steps, 1.0, 1e-10, 20000, lq.PRECISIONS[args.inner], 50)
        rows.append(r)
        print(json.dumps({"traj": traj, "dH": r["dH"], "accepted": r["accepted"], "plaquette": r["plaquette"],
                          "seconds": r["seconds"], "cg_iterations": r["cg_iterations"]}), flush=True)
    total = time.perf_counter() - t0
    lq.lq_destroy(ctx)
    half = rows[len(rows) // 2:]
    e = np.exp(-np.array([r["dH"] for r in half]))
    plaq = np.array([r["plaquette"] for r in half])
    dev_t = [r["seconds_solve"] + r["seconds_gauge_force"] + r["seconds_fermion_force"] + r["seconds_link_update"]
             for r in rows]
    share = {k: float(np.mean([r["seconds_" + k] / d for r, d in zip(rows, dev_t)]))
             for k in ("solve", "gauge_force", "fermion_force", "link_update")}
    print(json.dumps({"workload": "hmc_%dx%dx%dx%d" % dims, "start": args.start, "beta": args.beta,
                      "kappa": args.hmc_kappa, "md_steps": args.md_steps, "tau": 1.0, "inner": args.inner,
                      "trajectories": len(rows), "acceptance": float(np.mean([r["accepted"] for r in rows])),
                      "second_half": {"trajectories": len(half),
                                      "acceptance": float(np.mean([r["accepted"] for r in half])),
                                      "exp_minus_dH_mean": float(e.mean()),
                                      "exp_minus_dH_err": float(e.std() / np.sqrt(len(e))),
                                      "plaquette_mean": float(plaq.mean()),
                                      "plaquette_err": float(plaq.std() / np.sqrt(len(plaq)))},
                      "plaquette_last": rows[-1]["plaquette"],
                      "seconds_per_trajectory": float(np.mean([r["seconds"] for r in rows])),
                      "seconds_total": total,
                      "cg_iterations_per_trajectory": float(np.mean([r["cg_iterations"] for r in rows])),
                      "share": share}), flush=True)
    return 0


def run_reference(args):
    import numpy as np
    rank, size = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    lat, U, phi = make_inputs()
    n_iter = args.cg_iterations
    frac = args.ref_site_fraction
    for _ in range(args.warmup):
        oracle_cg_iteration_seconds(U, phi, frac)
    t = [oracle_cg_iteration_seconds(U, phi, frac) for _ in range(args.steps)]
    per_solve = float(np.mean(t)) * n_iter
    value = 1.0 / per_solve
    sample = ("one CG iteration of the FP64 oracle (M and M^dag on every %d-th site, scaled by %d, plus "
              "the vector updates on the full lattice) per step, times %d iterations (the FP64 CG "
              "iteration count of this workload)" % (frac, frac, n_iter))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": size,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3 / n_iter,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "dims": list(DIMS), "kappa": KAPPA,
                                            "sigma": SIGMA, "seed": SEED, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_kernel_only(args):
    """Profiling target: a few launches of one kernel (--kernel-only dslash|k1|k2|k3) in one precision."""
    import torch
    import paper_1207_2223_gb300 as lq
    from synth import Lattice, gauge_exp_iA, source
    dims = tuple(args.dims)
    lat = Lattice(dims)
    U, phi = gauge_exp_iA(lat, SIGMA, SEED), source(lat, SEED)
    ctx = lq.lq_create(dims)
    lq.lq_set_option(ctx, lq.LQ_OPT_PAIR_SITES, args.pair_sites)
    lq.lq_gauge_set(ctx, torch.from_numpy(U).cuda())
    p = torch.from_numpy(phi).cuda()
    prec = lq.PRECISIONS[args.prec]
    if args.kernel_only == "batch":
        import numpy as np
        R = 12
        phis = torch.from_numpy(np.stack([source(lat, SEED, i) for i in range(R)])).cuda()
        x = torch.zeros_like(phis)
        t0 = time.perf_counter()
        st = lq.lq_solve_batch([ctx], [x], [phis], [KAPPA], R, 1e-10, args.steps, prec, 50)
        lq.lq_destroy(ctx)
        print("batch %s %s x %d: %d iterations, %.4f s" % (args.prec, dims, R, st[1]["iterations"],
                                                          time.perf_counter() - t0))
        return 0
    if args.kernel_only == "dslash":
        ms = lq.lq_time_dslash(ctx, p, KAPPA, False, prec, args.steps, False)
    else:
        ms = lq.lq_time_cg_kernel(ctx, p, KAPPA, int(args.kernel_only[1]), prec, args.steps)
    lq.lq_destroy(ctx)
    print("%s %s %s: %.4f ms" % (args.kernel_only, args.prec, dims, ms))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import paper_1207_2223_gb300 as lq
    from paper_1207_2223_gb300 import replicas

    rank, size, local = replicas.world()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    dev = torch.device("cuda", local)
    inner = lq.PRECISIONS[args.inner]
    lat, U, phi = make_inputs()
    V = lat.V
    stream = torch.cuda.current_stream(dev)
    ctx = lq.lq_create(DIMS, True, stream.cuda_stream)
    try:
        Ud = torch.from_numpy(U).to(dev)
        lq.lq_gauge_set(ctx, Ud)
        phid = torch.from_numpy(phi).to(dev)
        x = torch.zeros_like(phid)

        def solve(prec, xo=x, ph=phid):
            status, st = lq.lq_solve_MdagM(ctx, xo, ph, KAPPA, TOL, 100000, prec, RELIABLE)
            if status != lq.LQ_OK or st["true_rel_resid"] > TOL:
                raise RuntimeError("solve failed: status %d %s" % (status, st))
            return st

        for _ in range(args.warmup):
            solve(inner)
        torch.cuda.synchronize(dev)
        replicas.barrier()
        clocks = Clocks(local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(solve(inner))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        replicas.barrier()
        t_local = e0.elapsed_time(e1) / 1e3
        t_job, units = replicas.combine(t_local, args.steps, dev)
        value = units / t_job
        launches = int(sum(s["kernel_launches"] for s in stats))

        # the other inner storage formats, one solve each (FP16-12 is the storage the
        # 32^3 x 64 workload names; FP32-12 is HBM-bound, the 16-bit formats issue-bound)
        others = {}
        for name in ("f32_12", "f16_12", "bf16_12", "i16_12"):
            if name == args.inner:
                continue
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            sto = solve(lq.PRECISIONS[name])
            q1.record(stream)
            torch.cuda.synchronize(dev)
            others[name] = {"seconds": q0.elapsed_time(q1) / 1e3, "iterations": sto["iterations"],
                            "reliable_updates": sto["reliable_updates"], "escalations": sto["escalations"]}

        # the same mixed solve with double-float intermediate reliable updates
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, 1)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        solve(inner)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        mixed_df_s = t0.elapsed_time(t1) / 1e3
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, 0)

        # plain FP64 CG on the same source: the comparison of the metric
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        st64 = solve(lq.LQ_F64)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_s = t0.elapsed_time(t1) / 1e3

        # kernels timed alone with CUDA events on the library's stream
        peaks, peak_kind = load_peaks()
        hbm = float(peaks["hbm_gbs"])
        dsl = {}
        for name in ("f64", "df64", "f32", "f32_12", "f16_12", "bf16_12", "i16_12"):
            ms = lq.lq_time_dslash(ctx, phid, KAPPA, False, lq.PRECISIONS[name], 20, False)
            gbs = DSLASH_BYTES[name] * V / (ms * 1e-3) / 1e9
            dsl[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                         "GFLOP/s": round(DSLASH_FLOPS * V / (ms * 1e-3) / 1e9, 1)}
        cg = {}
        for which in ("k1", "k2", "k3"):
            ms = lq.lq_time_cg_kernel(ctx, phid, KAPPA, int(which[1]), inner, 40)
            gbs = CG_BYTES[args.inner][which] * V / (ms * 1e-3) / 1e9
            cg[which] = {"ms": round(ms, 5), "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                         "bytes_per_site": CG_BYTES[args.inner][which]}
        cg["iteration_ms"] = round(lq.lq_time_cg_kernel(ctx, phid, KAPPA, 0, inner, 40), 5)
        # the two-site packed FP32x2 variant of the 16-bit passes (LQ_OPT_PAIR_SITES, off by
        # default: fewer instructions, same FMA-pipe time, lower occupancy)
        # (16-bit fixed point only), against the one-site passes of the same format
        i16 = lq.LQ_I16_12
        two_site = {"one_site": {w: round(lq.lq_time_cg_kernel(ctx, phid, KAPPA, int(w[1]), i16, 40), 5)
                                 for w in ("k1", "k2")}}
        lq.lq_set_option(ctx, lq.LQ_OPT_PAIR_SITES, 1)
        two_site.update({w: round(lq.lq_time_cg_kernel(ctx, phid, KAPPA, int(w[1]), i16, 40), 5)
                         for w in ("k1", "k2")})
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        sto = solve(i16)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        two_site["solve_s"] = q0.elapsed_time(q1) / 1e3
        two_site["iterations"] = sto["iterations"]
        lq.lq_set_option(ctx, lq.LQ_OPT_PAIR_SITES, 0)
        src_hash = kernel_source_hash()
        tr = NCU_TRAFFIC.get(args.inner)
        traffic = tr["bytes_per_site"] * V if tr and tr.get("src") == src_hash else None
        d = cg["k2"]
        # the dominant kernel of the timed step (largest share of the launch list):
        # CG pass 2, r -= alpha M^dag t, x += alpha p, |r|^2
        roofline = {"kernel": "dslash_kernel<%s, M^dag, EpiCG2> (CG pass 2)" % args.inner, "bound": "hbm",
                    "achieved": d["GB/s"], "peak": hbm, "unit": "GB/s", "frac": d["frac_hbm"],
                    "traffic": traffic, "peak_kind": peak_kind,
                    "bytes_per_site": CG_BYTES[args.inner]["k2"], "sites_per_launch": V,
                    "launch_ms": d["ms"]}

        # end to end through the C interface with pinned host buffers
        Uh = torch.from_numpy(U).pin_memory()
        phih = torch.from_numpy(phi).pin_memory()
        xh = torch.empty_like(phih).pin_memory()
        lq.lq_gauge_set(ctx, Uh)
        solve(inner, xh, phih)
        clocks_e2e = Clocks(local)
        t_set, t_solve = [], []
        t_e = time.perf_counter()
        for _ in range(args.steps):
            ta = time.perf_counter()
            lq.lq_gauge_set(ctx, Uh)
            tb = time.perf_counter()
            solve(inner, xh, phih)
            t_set.append(tb - ta)
            t_solve.append(time.perf_counter() - tb)
        e2e_local = time.perf_counter() - t_e
        clk_e2e = clocks_e2e.stop()
        e2e_t, e2e_units = replicas.combine(e2e_local, args.steps, dev)
        e2e = {"value": e2e_units / e2e_t, "unit": "solves/s", "h2d_bytes_per_step": int(U.nbytes + phi.nbytes),
               "d2h_bytes_per_step": int(phi.nbytes),
               "gauge_set_ms": round(1e3 * sorted(t_set)[len(t_set) // 2], 2),
               "solve_ms": round(1e3 * sorted(t_solve)[len(t_solve) // 2], 2), "clocks": clk_e2e}
        # host <-> device copy rate of pinned buffers (context for e2e)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        Ud.copy_(Uh, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        h2d = U.nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9
        c0.record(stream)
        Uh.copy_(Ud, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        e2e["pinned_copy_gbs"] = {"h2d": h2d, "d2h": U.nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9}

        extras = None if args.no_extras else measure_extras(lq, torch, dev)

        cpu = None
        if rank == 0 and size == 1 and not args.no_cpu:
            t_it = oracle_cg_iteration_seconds(U, phi, args.ref_site_fraction)
            n_it = st64["iterations"]
            cpu = {"value": 1.0 / (t_it * n_it), "unit": "solves/s", "cores": 1, "kind": "oracle",
                   "sample": "one CG iteration of the FP64 oracle (M and M^dag on every %d-th site, scaled, "
                             "plus the vector updates), times the %d iterations of the FP64 CG"
                             % (args.ref_site_fraction, n_it),
                   "seconds_per_iteration": t_it}
    finally:
        lq.lq_destroy(ctx)

    mixed_s = t_local / args.steps
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": size, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_job / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if inner != lq.LQ_F64 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "kappa": KAPPA, "sigma": SIGMA, "seed": SEED,
                       "tol": TOL, "inner": args.inner, "reliable_every": RELIABLE,
                       "l2": "working set larger than L2 (gauge %d MB + spinors), no flush"
                             % (DSLASH_BYTES[args.inner] * V // 3 // 2**20),
                       "parallelism": "replicas" if size > 1 else "single"},
            "time_to_solution_s": {"mixed": mixed_s, "fp64": fp64_s, "speedup": fp64_s / mixed_s,
                                   "mixed_double_float_reliable_updates": mixed_df_s,
                                   "other_inner_formats": others},
            "iterations": {"mixed": stats[-1]["iterations"], "reliable_updates": stats[-1]["reliable_updates"],
                           "fp64": st64["iterations"]},
            "true_rel_resid": {"mixed": stats[-1]["true_rel_resid"], "fp64": st64["true_rel_resid"]},
            "roofline": roofline, "cg_kernels": cg, "cg_kernels_two_site": two_site, "dslash": dsl, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if extras is not None:
        line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--inner", default="f16_12", choices=["f32", "f32_12", "f16_12", "bf16_12", "i16_12"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true", help="skip the HMC, batch and iteration-scan numbers")
    ap.add_argument("--ref-site-fraction", type=int, default=8)
    ap.add_argument("--cg-iterations", type=int, default=312,
                    help="FP64 CG iterations of this workload (reference arm extrapolation)")
    ap.add_argument("--kernel-only", default=None, choices=["dslash", "k1", "k2", "k3", "batch"],
                    help="profiling target: only launch this kernel (precision --prec); batch: a 12-RHS "
                         "batched solve of --steps iterations")
    ap.add_argument("--prec", default="f32_12", choices=["f64", "f32", "f32_12", "f16_12", "bf16_12", "i16_12"])
    ap.add_argument("--dims", type=int, nargs=4, default=list(DIMS))
    ap.add_argument("--md-steps", type=int, default=25, help="leapfrog steps per trajectory (--hmc-ensemble)")
    ap.add_argument("--trajectories", type=int, default=20, help="--hmc-ensemble: number of trajectories")
    ap.add_argument("--beta", type=float, default=5.7, help="--hmc-ensemble: gauge coupling")
    ap.add_argument("--hmc-kappa", type=float, default=0.155, help="--hmc-ensemble: hopping parameter")
    ap.add_argument("--start", choices=["exp", "ordered"], default="exp",
                    help="--hmc-ensemble: exp(iA) start (sigma 0.3, seed 8) or ordered start U = 1")
    ap.add_argument("--pair-sites", type=int, default=0, choices=[0, 1],
                    help="--kernel-only: two-site packed stencil for i16_12 (LQ_OPT_PAIR_SITES)")
    ap.add_argument("--hmc-ensemble", action="store_true",
                    help="run --steps HMC trajectories at 32^4 (beta 5.7, kappa 0.155, 25 steps) and report "
                         "acceptance and <exp(-dH)> instead of the benchmark")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_only:
        return run_kernel_only(args)
    if args.hmc_ensemble:
        return run_hmc_ensemble(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
