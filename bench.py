#!/usr/bin/env python
"""Benchmark of the hot path: CG time-to-1e-10 and Dslash bandwidth at 32^3 x 64.

Workload (synthetic, seeded): a 32^3 x 64 SU(3) lattice with links
U = exp(iA), A traceless Hermitian with N(0, 0.25^2) entries (seed 2),
kappa = 0.156, antiperiodic time, a complex Gaussian source; M^dag M x = phi
is solved from x0 = 0 to an FP64 true relative residual of 1e-10.

One step = one mixed-precision solve (inner precision --inner, default FP16
storage with 12-real links and per-site FP32 norms, FP32 arithmetic, reliable
updates every 50 iterations: the intermediate ones in double-float arithmetic,
the last recomputed and certified in FP64; the all-FP64-update solve is
reported beside it).  Printed as one JSON line:
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
# DRAM traffic per site of CG pass 2 (r -= alpha M^dag t, x += alpha p, |r|^2) from one
# ncu capture per storage format: dram__bytes_read.sum + dram__bytes_write.sum of a
# single launch on a 32^4 lattice, divided by its 1,048,576 sites.  Valid for the kernel
# sources with this hash; null once the kernel has changed since the capture.
NCU_TRAFFIC = {
    "f16_12": {"bytes_per_site": 466.1, "src": "a4d74c9cc5d7204c"},
}


def kernel_source_hash():
    """Hash of the code (comments and blank space removed) of the device code of the CG
    passes, so that a comment or host-side edit does not void the traffic figures."""
    import re
    h = hashlib.sha256()
    for f in ("lq_device.cuh", "lq_df64.cuh", "lq_dslash.cuh", "k_cglo.cu"):
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


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ---- the FP64 oracle's CG, timed on the host cores (cpu_baseline and the reference arm)
# Worker processes (started with spawn, never forked from a process that touched the GPU)
# attach to the gauge field and the CG vectors in shared memory and each evaluates the
# oracle's M or M^dag (oracle.wilson.apply_M, unchanged) on one slab of output sites.
_W = {}


def _oracle_worker_init(names, V, dims, kappa):
    import numpy as np
    from multiprocessing import shared_memory
    from oracle.conventions import neighbours
    _W["shm"] = {k: shared_memory.SharedMemory(name=n) for k, n in names.items()}
    shape = {"U": (V, 4, 3, 3)}
    _W["a"] = {k: np.ndarray(shape.get(k, (V, 4, 3)), dtype=np.complex128, buffer=m.buf)
               for k, m in _W["shm"].items()}
    _W["nbr"] = neighbours(dims, True)
    _W["dims"], _W["kappa"] = dims, kappa


def _oracle_worker_apply(job):
    import numpy as np
    from oracle.wilson import apply_M
    src, dst, lo, hi, dagger = job
    a = _W["a"]
    a[dst][lo:hi] = apply_M(a["U"], a[src], _W["dims"], _W["kappa"], True, dagger, np.arange(lo, hi), _W["nbr"])
    return hi - lo


class OracleCG:
    """Textbook CG on M^dag M with the FP64 oracle's operator, from x0 = 0, one iteration per
    step().  With nproc > 1 each application of M / M^dag runs on nproc slabs of sites in a
    process pool; the vector updates run in this process."""

    def __init__(self, U, phi, nproc):
        import numpy as np
        self.np = np
        self.V = U.shape[0]
        self.nproc = nproc
        self.pool = None
        self.shm = []
        if nproc > 1:
            import multiprocessing as mp
            from multiprocessing import shared_memory
            names, arr = {}, {}
            for k, like in (("U", U), ("p", phi), ("t", phi), ("s", phi)):
                m = shared_memory.SharedMemory(create=True, size=like.nbytes)
                self.shm.append(m)
                names[k] = m.name
                arr[k] = np.ndarray(like.shape, dtype=np.complex128, buffer=m.buf)
            arr["U"][...] = U
            self.a = arr
            self.pool = mp.get_context("spawn").Pool(nproc, initializer=_oracle_worker_init,
                                                     initargs=(names, self.V, DIMS, KAPPA))
            self.pool.map(_oracle_worker_apply, [("p", "t", 0, 1, False)] * nproc)   # start every worker
            edges = np.linspace(0, self.V, nproc + 1).astype(int)
            self.slabs = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]
        else:
            from oracle.conventions import neighbours
            self.nbr = neighbours(DIMS, True)
            self.a = {"U": U, "p": phi.copy(), "t": np.empty_like(phi), "s": np.empty_like(phi)}
        self.x = np.zeros_like(phi)
        self.r = phi.copy()
        self.a["p"][...] = phi
        self.rr = float(np.vdot(self.r, self.r).real)
        self.phi2 = self.rr

    def _apply(self, src, dst, dagger):
        if self.pool is not None:
            self.pool.map(_oracle_worker_apply, [(src, dst, lo, hi, dagger) for lo, hi in self.slabs])
        else:
            from oracle.wilson import apply_M
            self.a[dst][...] = apply_M(self.a["U"], self.a[src], DIMS, KAPPA, True, dagger, None, self.nbr)

    def step(self):
        """One CG iteration; returns its wall-clock seconds."""
        np = self.np
        t0 = time.perf_counter()
        self._apply("p", "t", False)               # t = M p
        self._apply("t", "s", True)                # s = M^dag t = M^dag M p
        p, t, s = self.a["p"], self.a["t"], self.a["s"]
        alpha = self.rr / float(np.vdot(t, t).real)
        self.x += alpha * p
        self.r -= alpha * s
        rr_new = float(np.vdot(self.r, self.r).real)
        p *= rr_new / self.rr
        p += self.r
        self.rr = rr_new
        return time.perf_counter() - t0

    def rel_residual(self):
        return (self.rr / self.phi2) ** 0.5

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        self.a = None
        for m in self.shm:
            m.close()
            m.unlink()
        self.shm = []


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sampled_residual(U, phi, x, n_sites=200, seed=0):
    """FP64 true relative residual of a solution x at sampled sites, evaluated by the oracle
    (M^dag M x at each sampled site from its one-hop neighbourhood), relative to phi there."""
    import numpy as np
    from oracle.wilson import apply_MdagM_sites
    V = U.shape[0]
    rng = np.random.default_rng(seed)
    sites = np.unique(np.concatenate([rng.integers(0, V, n_sites), [0, V - 1]]))
    Ax = apply_MdagM_sites(U, x, DIMS, KAPPA, sites)
    r = phi[sites] - Ax
    return float(np.linalg.norm(r) / np.linalg.norm(phi[sites])), int(len(sites))


def hmc_chain(lq, torch, dev, dims, U, seed, n_traj, beta, kappa, steps, prec):
    """n_traj HMC trajectories in one context from links U (device), with the heat bath
    (momenta, noise, Metropolis uniform) drawn on the device from the generator's streams
    (trajectories 0 .. n_traj - 1 of `seed`).  Returns a summary."""
    import numpy as np
    rows = []
    ctx = lq.lq_create(dims, True, torch.cuda.current_stream(dev).cuda_stream)
    try:
        lq.lq_gauge_set(ctx, U)
        for traj in range(n_traj):
            rows.append(lq.lq_hmc_trajectory_seeded(ctx, seed, traj, beta, kappa, steps, 1.0, 1e-10, 20000, prec, 50))
    finally:
        lq.lq_destroy(ctx)
    dev_t = [r["seconds_solve"] + r["seconds_gauge_force"] + r["seconds_fermion_force"] + r["seconds_link_update"]
             for r in rows]
    dh = np.array([r["dH"] for r in rows])
    sec = np.array([r["seconds"] for r in rows])
    return {"trajectories": n_traj, "seconds_per_trajectory": float(sec.mean()),
            "trajectories_per_s": float(n_traj / sec.sum()), "dH": [float(v) for v in dh],
            "acceptance": float(np.mean([r["accepted"] for r in rows])),
            # undefined (overflows) while a chain still falls from a rough start with dH << 0
            "exp_minus_dH_mean": float(np.mean(np.exp(-dh))) if np.all(dh > -700.0) else None,
            "plaquette": [float(r["plaquette"]) for r in rows],
            "cg_iterations_per_trajectory": float(np.mean([r["cg_iterations"] for r in rows])),
            "solves_per_trajectory": rows[0]["solves"],
            "share": {k: float(np.mean([r["seconds_" + k] / d for r, d in zip(rows, dev_t)]))
                      for k in ("solve", "gauge_force", "fermion_force", "link_update")}}


def measure_extras(lq, torch, dev):
    """Numbers beside the headline, each measured once outside the timed region: the
    other workloads (one trajectory at 4^4; 1000 operator applications, a solve and 5
    trajectories at 16^4; trajectories at 32^4; the differentiable action at 16^4), the
    per-routine split of trajectories across volumes, the batched solve at 24^4 x 12,
    the register ablation, and CG time against iteration count with and without CUDA
    graphs (per-call overhead = intercept)."""
    import numpy as np
    from synth import Lattice, gauge_exp_iA, source
    out = {}
    # one plain FP64 trajectory at 4^4 (beta 5.6, kappa 0.15, 10 steps, tau 1, sigma 0.3, seed 0)
    lat = Lattice((4, 4, 4, 4))
    U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 0)).to(dev)
    out["hmc_4x4x4x4_f64"] = hmc_chain(lq, torch, dev, (4, 4, 4, 4), U, 0, 1, 5.6, 0.15, 10, lq.LQ_F64)
    # 16^4 (sigma 0.3, seed 1, reunitarised, kappa 0.155): 1000 applications of M in FP64 and
    # FP32 (the lattice fits in L2), one solve to 1e-10, 5 trajectories (beta 5.6, 20 steps)
    dims = (16, 16, 16, 16)
    lat = Lattice(dims)
    V16 = lat.V
    U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 1, reunitarise=True)).to(dev)
    phi = torch.from_numpy(source(lat, 1)).to(dev)
    c2 = {}
    ctx = lq.lq_create(dims, True, torch.cuda.current_stream(dev).cuda_stream)
    try:
        lq.lq_gauge_set(ctx, U)
        for name in ("f64", "f32"):
            ms = lq.lq_time_dslash(ctx, phi, 0.155, False, lq.PRECISIONS[name], 1000, False)
            c2["dslash_1000_" + name] = {"ms_per_application": ms,
                                         "GB/s": DSLASH_BYTES[name] * V16 / (ms * 1e-3) / 1e9,
                                         "GFLOP/s": DSLASH_FLOPS * V16 / (ms * 1e-3) / 1e9}
        for name in ("f64", "f32", "f16_12"):
            x = torch.zeros_like(phi)
            t0 = time.perf_counter()
            _, st = lq.lq_solve_MdagM(ctx, x, phi, 0.155, 1e-10, 20000, lq.PRECISIONS[name], 50)
            c2["solve_" + name] = {"seconds": time.perf_counter() - t0, "iterations": st["iterations"],
                                   "true_rel_resid": st["true_rel_resid"]}
    finally:
        lq.lq_destroy(ctx)
    for name in ("f64", "f32", "f16_12"):
        c2["hmc_5traj_" + name] = hmc_chain(lq, torch, dev, dims, U, 1, 5, 5.6, 0.155, 20, lq.PRECISIONS[name])
    out["wilson_16x16x16x16"] = c2
    # per-routine split of a trajectory (mixed FP16-12 solves) at 8^4 and 24^4, same parameters
    for d in (8, 24):
        dims = (d, d, d, d)
        lat = Lattice(dims)
        U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 1, reunitarise=True)).to(dev)
        out["hmc_%dx%dx%dx%d_f16_12" % dims] = hmc_chain(lq, torch, dev, dims, U, 1, 1, 5.6, 0.155, 20,
                                                         lq.LQ_F16_12)
    # 32^4 trajectories of the differentiable-action workload (beta 5.7, kappa 0.155, 25 steps,
    # tau 1, mixed FP16-12 solves, exp(iA) start sigma 0.3 seed 8): the first 3 of its 20
    dims = (32, 32, 32, 32)
    lat = Lattice(dims)
    U = torch.from_numpy(gauge_exp_iA(lat, 0.3, 8)).to(dev)
    out["hmc_32x32x32x32_f16_12"] = hmc_chain(lq, torch, dev, dims, U, 8, 3, 5.7, 0.155, 25, lq.LQ_F16_12)
    del U
    # differentiable S_f at 16^4 (kappa 0.15, seed 8): forward + backward per step through the
    # cached context (the first step creates it and records the solver's CUDA graphs)
    from paper_1207_2223_gb300 import autograd as ag
    dims = (16, 16, 16, 16)
    lat = Lattice(dims)
    Ua = torch.from_numpy(gauge_exp_iA(lat, 0.3, 8)).to(dev).requires_grad_(True)
    phia = torch.from_numpy(source(lat, 8)).to(dev)
    ag.release_contexts()
    steps_s = []
    for _ in range(6):
        Ua.grad = None
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ag.pseudofermion_action(Ua, phia, dims, 0.15, 1e-10).backward()
        torch.cuda.synchronize(dev)
        steps_s.append(time.perf_counter() - t0)
    out["autograd_16x16x16x16"] = {"first_step_s": steps_s[0], "step_s": float(np.median(steps_s[1:])),
                                   "gauge_loads": list(ag.cached_context_stats().values())[0]}
    ag.release_contexts()
    del Ua, phia
    # batched solves: (a) 24^4, kappa 0.155, seed 3, 12 right-hand sides sharing one gauge
    # field; (b) lattices 8^4, 12^4, 16^4, 8^3 x 16 with kappa 0.12 .. 0.155, seeds 4-7.  Per
    # shape: the autotuned per-pass launches and the persistent launch, against the same
    # systems solved one after another; per-column residual histories (every 25th iteration)
    def batch(shapes, kappas, seeds, R, prec):
        ctxs, xs, phs = [], [], []
        for d, sd in zip(shapes, seeds):
            lt = Lattice(d)
            cx = lq.lq_create(d, True, torch.cuda.current_stream(dev).cuda_stream)
            lq.lq_gauge_set(cx, torch.from_numpy(gauge_exp_iA(lt, 0.3, sd)).to(dev))
            ctxs.append(cx)
            src = np.stack([source(lt, sd, i) for i in range(R)]) if R > 1 else source(lt, sd)
            phs.append(torch.from_numpy(src).to(dev))
            xs.append(torch.zeros_like(phs[-1]))
        res = {}
        try:
            # the whole solve as one graph with conditional nodes (default), one graph per
            # chunk of iterations with the decisions on the host, one persistent launch per chunk
            for form, pers, loop in (("device_loop", 0, 1), ("host_loop", 0, 0), ("persistent", 1, 0)):
                lq.lq_set_option(ctxs[0], lq.LQ_OPT_BATCH_PERSISTENT, pers)
                lq.lq_set_option(ctxs[0], lq.LQ_OPT_BATCH_DEVICE_LOOP, loop)
                lq.lq_solve_batch(ctxs, xs, phs, kappas, R, 1e-10, 20000, prec, 50)       # tunes, records
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                status, st, iters, resid, hist = lq.lq_solve_batch(ctxs, xs, phs, kappas, R, 1e-10, 20000, prec,
                                                                   50, hist_len=4000)
                torch.cuda.synchronize(dev)
                res[form] = {
                    "seconds": time.perf_counter() - t0, "iterations": st["iterations"],
                    "reliable_updates": st["reliable_updates"], "kernel_launches": st["kernel_launches"],
                    "max_true_rel_resid": float(resid.max()), "column_iterations": [int(v) for v in iters]}
            res["tuning"] = lq.lq_batch_tuning(ctxs[0])
            res["residual_history_every_25"] = [[float("%.3e" % v) for v in h[:st["iterations"]:25]] for h in hist]
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for cx, ph, k in zip(ctxs, phs, kappas):
                for i in range(R):
                    rhs = ph[i] if R > 1 else ph
                    lq.lq_solve_MdagM(cx, torch.zeros_like(rhs), rhs, k, 1e-10, 20000, prec, 50)
            torch.cuda.synchronize(dev)
            res["sequential_seconds"] = time.perf_counter() - t0
            best = min(res[f]["seconds"] for f in ("device_loop", "host_loop", "persistent"))
            res["speedup_vs_sequential"] = res["sequential_seconds"] / best
        finally:
            for cx in ctxs:
                lq.lq_destroy(cx)
        return res
    out["batch_24x24x24x24_12rhs_f16_12"] = batch([(24, 24, 24, 24)], [0.155], [3], 12, lq.LQ_F16_12)
    out["batch_24x24x24x24_12rhs_f32_12"] = batch([(24, 24, 24, 24)], [0.155], [3], 12, lq.LQ_F32_12)
    out["batch_uneven_f16_12"] = batch([(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (8, 8, 8, 16)],
                                       [0.12, 0.14, 0.15, 0.155], [4, 5, 6, 7], 1, lq.LQ_F16_12)
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
    from synth import Lattice, gauge_exp_iA, identity_gauge
    dims = tuple(args.dims) if tuple(args.dims) != DIMS else (32, 32, 32, 32)
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    U0 = identity_gauge(lat) if args.start == "ordered" else gauge_exp_iA(lat, 0.3, 8)
    lq.lq_gauge_set(ctx, torch.from_numpy(U0).cuda())
    rows = []
    t0 = time.perf_counter()
    for traj in range(args.trajectories):
        r = lq.lq_hmc_trajectory_seeded(ctx, 8, traj, args.beta, args.hmc_kappa, args.md_steps, 1.0, 1e-10, 20000,
                                        lq.PRECISIONS[args.inner], 50)
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


def oracle_timing(U, phi, all_steps, warmup, single_steps):
    """Time the FP64 oracle's CG on this host: `warmup` + `all_steps` iterations on every core
    (process pool over site slabs), then `single_steps` iterations on one core.  Returns a
    dict with the per-step times and the host description."""
    import numpy as np
    n = host_cores()
    out = {"cores": n, "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    cg = OracleCG(U, phi, n)
    try:
        for _ in range(warmup):
            cg.step()
        t = [cg.step() for _ in range(all_steps)]
        out["all_cores_s_per_iteration"] = t
        out["all_cores_rel_residual_after"] = cg.rel_residual()
    finally:
        cg.close()
    if single_steps > 0:
        cg1 = OracleCG(U, phi, 1)
        out["single_core_s_per_iteration"] = [cg1.step() for _ in range(single_steps)]
        cg1.close()
    out["iterations_done"] = warmup + all_steps
    out["median_all"] = float(np.median(t)) if t else None
    return out


# FP64 CG iterations of the 32^3 x 64 workload to a 1e-10 true residual (measured with
# the plain FP64 GPU CG, which follows the same algorithm from the same x0 = 0)
FP64_ITERATIONS = 312


def run_reference(args):
    """The reference arm: the project's FP64 CPU oracle (written from the paper), as it stands,
    on the host cores.  One step = one full CG iteration of the oracle on the whole 32^3 x 64
    lattice (M and M^dag on all sites over a process pool, vector updates in the main
    process); solves/s = 1 / (measured time per iteration x the FP64 iteration count)."""
    import numpy as np
    rank, size = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    lat, U, phi = make_inputs()
    tm = oracle_timing(U, phi, args.steps, args.warmup, 1 if args.single_core else 0)
    t_it = tm["median_all"]
    value = 1.0 / (t_it * FP64_ITERATIONS)
    sample = ("one full FP64 CG iteration of the oracle per step (M and M^dag on all %d sites on %d host "
              "processes, vector updates in one), solves/s = 1 / (median time per iteration x %d, the "
              "iteration count of the FP64 CG on this workload)" % (lat.V, tm["cores"], FP64_ITERATIONS))
    cpu = {"value": value, "unit": "solves/s", "cores": tm["cores"], "kind": "oracle", "sample": sample,
           "cpu_model": tm["cpu_model"], "nproc": tm["nproc"],
           "seconds_per_iteration_all_cores": t_it,
           "iterations_per_solve": FP64_ITERATIONS}
    if tm.get("single_core_s_per_iteration"):
        t1 = float(np.median(tm["single_core_s_per_iteration"]))
        cpu["single_core"] = {"seconds_per_iteration": t1, "value": 1.0 / (t1 * FP64_ITERATIONS),
                              "unit": "solves/s"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": size,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "dims": list(DIMS), "kappa": KAPPA,
                                            "sigma": SIGMA, "seed": SEED, "tol": TOL},
            "step": "one FP64 CG iteration of the oracle; value = solves/s = 1 / (ms_per_step x %d)"
                    % FP64_ITERATIONS,
            "iterations_per_solve": FP64_ITERATIONS,
            "cpu_baseline": cpu,
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
    lq.lq_set_option(ctx, lq.LQ_OPT_STAGED, args.staged)
    lq.lq_gauge_set(ctx, torch.from_numpy(U).cuda())
    p = torch.from_numpy(phi).cuda()
    prec = lq.PRECISIONS[args.prec]
    if args.kernel_only == "batch":
        import numpy as np
        R = 12
        # the profiled passes are the inner-format iterations; FP64 reliable updates keep the
        # device footprint small (no double-float fields)
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, 0)
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
        x_mixed = x.cpu().numpy()             # the timed solves' solution (checked by the oracle below)

        # the other inner storage formats, one solve each (FP16-12 is the storage the
        # 32^3 x 64 workload names; FP32-12 is HBM-bound, the 16-bit formats issue-bound)
        others = {}
        for name in ("f32_12", "f16_12", "bf16_12", "i16_12"):
            if name == args.inner:
                continue
            solve(lq.PRECISIONS[name])            # first solve of a format: fields, links, graphs
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            sto = solve(lq.PRECISIONS[name])
            q1.record(stream)
            torch.cuda.synchronize(dev)
            others[name] = {"seconds": q0.elapsed_time(q1) / 1e3, "iterations": sto["iterations"],
                            "reliable_updates": sto["reliable_updates"], "escalations": sto["escalations"]}

        # the same mixed solve with every reliable update in FP64 (the default does the
        # intermediate ones in double-float arithmetic and certifies the last in FP64)
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, 0)
        solve(inner)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        st_fp64ru = solve(inner)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        mixed_fp64ru_s = t0.elapsed_time(t1) / 1e3
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, 1)

        # plain FP64 CG on the same source: the comparison of the metric
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        st64 = solve(lq.LQ_F64)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_s = t0.elapsed_time(t1) / 1e3
        x_fp64 = x.cpu().numpy()

        # kernels timed alone with CUDA events on the library's stream
        peaks, peak_kind = load_peaks()
        hbm = float(peaks["hbm_gbs"])
        dsl = {}
        for name in ("f64", "df64", "f32", "f32_12", "f16_12", "bf16_12", "i16_12"):
            ms = lq.lq_time_dslash(ctx, phid, KAPPA, False, lq.PRECISIONS[name], 20, False)
            gbs = DSLASH_BYTES[name] * V / (ms * 1e-3) / 1e9
            dsl[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                         "GFLOP/s": round(DSLASH_FLOPS * V / (ms * 1e-3) / 1e9, 1)}
        # the FP64 operator is bound by the FP64 pipe: its roofline is the measured FP64
        # fused multiply-add rate of this GPU (FP32 rate for comparison)
        fma = {"f64_tflops": lq.lq_time_fma_peak(ctx, lq.LQ_F64), "f32_tflops": lq.lq_time_fma_peak(ctx, lq.LQ_F32)}
        d64 = dsl["f64"]
        fp64_roofline = {"kernel": "dslash_kernel<f64> (M)", "bound": "alu",
                         "achieved": round(d64["GFLOP/s"] / 1e3, 4), "peak": round(fma["f64_tflops"], 4),
                         "unit": "TFLOP/s", "frac": round(d64["GFLOP/s"] / 1e3 / fma["f64_tflops"], 4),
                         "peak_kind": "measured (lq_time_fma_peak: FP64 fused multiply-add chains)",
                         "flop_per_site": DSLASH_FLOPS, "launch_ms": d64["ms"]}
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
        t_set, t_solve, phases = [], [], []
        t_e = time.perf_counter()
        for _ in range(args.steps):
            ta = time.perf_counter()
            lq.lq_gauge_set(ctx, Uh)
            tb = time.perf_counter()
            st_e = solve(inner, xh, phih)
            t_set.append(tb - ta)
            t_solve.append(time.perf_counter() - tb)
            phases.append((st_e["stage_ms"], st_e["solve_ms"], st_e["deliver_ms"]))
        e2e_local = time.perf_counter() - t_e
        clk_e2e = clocks_e2e.stop()
        e2e_t, e2e_units = replicas.combine(e2e_local, args.steps, dev)
        e2e = {"value": e2e_units / e2e_t, "unit": "solves/s", "h2d_bytes_per_step": int(U.nbytes + phi.nbytes),
               "d2h_bytes_per_step": int(phi.nbytes),
               "gauge_set_ms": round(1e3 * sorted(t_set)[len(t_set) // 2], 2),
               "solve_ms": round(1e3 * sorted(t_solve)[len(t_solve) // 2], 2), "clocks": clk_e2e,
               # device time of the call's phases (CUDA events on its stream), median step
               "call_phases_ms": dict(zip(("stage_in", "solve", "deliver"),
                                          [round(sorted(p[i] for p in phases)[len(phases) // 2], 2)
                                           for i in range(3)]))}
        # host <-> device copy rate of pinned buffers through the copy engines (context for
        # e2e, which reads and writes the pinned buffers in place): median and slowest of 5
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rates = {"h2d": [], "d2h": []}
        for _ in range(5):
            for kind, (dst, src) in (("h2d", (Ud, Uh)), ("d2h", (Uh, Ud))):
                c0.record(stream)
                dst.copy_(src, non_blocking=True)
                c1.record(stream)
                torch.cuda.synchronize(dev)
                rates[kind].append(U.nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9)
        e2e["pinned_copy_gbs"] = {k: {"median": round(sorted(v)[2], 1), "slowest": round(min(v), 1)}
                                  for k, v in rates.items()}

        extras = None if args.no_extras else measure_extras(lq, torch, dev)

        cpu = None
        if rank == 0 and size == 1 and not args.no_cpu:
            # the oracle on the host cores: a bounded sample of its FP64 CG on this workload
            tm = oracle_timing(U, phi, 3, 1, 1)
            t_all = tm["median_all"]
            t_one = float(tm["single_core_s_per_iteration"][0])
            n_it = st64["iterations"]
            cpu = {"value": 1.0 / (t_all * n_it), "unit": "solves/s", "cores": tm["cores"], "kind": "oracle",
                   "sample": "4 full FP64 CG iterations of the oracle (M and M^dag on all %d sites over %d host "
                             "processes; the first untimed), median time per iteration x the %d iterations "
                             "of the FP64 CG; then one iteration on a single core" % (V, tm["cores"], n_it),
                   "cpu_model": tm["cpu_model"], "nproc": tm["nproc"],
                   "seconds_per_iteration_all_cores": t_all,
                   "single_core": {"seconds_per_iteration": t_one, "value": 1.0 / (t_one * n_it),
                                   "unit": "solves/s"}}
            # the oracle's own FP64 residual of the GPU solutions at sampled sites (config
            # 3: FP64 oracle error reported for the solution)
            check = {}
            for name, xs in (("mixed", x_mixed), ("fp64", x_fp64)):
                rel, ns = oracle_sampled_residual(U, phi, xs)
                check[name] = rel
            check["sites"] = ns
            cpu["oracle_residual_of_gpu_solution"] = check
    finally:
        lq.lq_destroy(ctx)

    mixed_s = t_local / args.steps
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": size, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_job / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if inner != lq.LQ_F64 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "kappa": KAPPA, "sigma": SIGMA, "seed": SEED,
                       "tol": TOL, "inner": args.inner, "reliable_every": RELIABLE,
                       "reliable_updates": "intermediate in double-float (FP32 pipe, ~48 bits), the last "
                                           "recomputed and certified in FP64",
                       "l2": "working set larger than L2 (gauge %d MB + spinors), no flush"
                             % (DSLASH_BYTES[args.inner] * V // 3 // 2**20),
                       "parallelism": "replicas" if size > 1 else "single"},
            "time_to_solution_s": {"mixed": mixed_s, "fp64": fp64_s, "speedup": fp64_s / mixed_s,
                                   "mixed_fp64_reliable_updates": {"seconds": mixed_fp64ru_s,
                                                                   "iterations": st_fp64ru["iterations"],
                                                                   "reliable_updates": st_fp64ru["reliable_updates"]},
                                   "other_inner_formats": others},
            "iterations": {"mixed": stats[-1]["iterations"], "reliable_updates": stats[-1]["reliable_updates"],
                           "fp64": st64["iterations"]},
            "true_rel_resid": {"mixed": stats[-1]["true_rel_resid"], "fp64": st64["true_rel_resid"]},
            "roofline": roofline, "fp64_roofline": fp64_roofline, "fma_peaks": fma, "cg_kernels": cg, "cg_kernels_two_site": two_site, "dslash": dsl, "e2e": e2e,
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
    ap.add_argument("--single-core", type=int, default=1, choices=[0, 1],
                    help="--impl reference: also time one oracle CG iteration on a single core")
    ap.add_argument("--kernel-only", default=None, choices=["dslash", "k1", "k2", "k3", "batch"],
                    help="profiling target: only launch this kernel (precision --prec); batch: a 12-RHS "
                         "batched solve of --steps iterations")
    ap.add_argument("--prec", default="f32_12", choices=["f64", "df64", "f32", "f32_12", "f16_12", "bf16_12", "i16_12"])
    ap.add_argument("--dims", type=int, nargs=4, default=list(DIMS))
    ap.add_argument("--md-steps", type=int, default=25, help="leapfrog steps per trajectory (--hmc-ensemble)")
    ap.add_argument("--trajectories", type=int, default=20, help="--hmc-ensemble: number of trajectories")
    ap.add_argument("--beta", type=float, default=5.7, help="--hmc-ensemble: gauge coupling")
    ap.add_argument("--hmc-kappa", type=float, default=0.155, help="--hmc-ensemble: hopping parameter")
    ap.add_argument("--start", choices=["exp", "ordered"], default="exp",
                    help="--hmc-ensemble: exp(iA) start (sigma 0.3, seed 8) or ordered start U = 1")
    ap.add_argument("--pair-sites", type=int, default=0, choices=[0, 1],
                    help="--kernel-only: two-site packed stencil for i16_12 (LQ_OPT_PAIR_SITES)")
    ap.add_argument("--staged", type=int, default=0, choices=[0, 1],
                    help="--kernel-only: the stencil sharing x and y links in-block (LQ_OPT_STAGED)")
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
