"""Benchmark: ms per midpoint time step of the time-dependent Hubbard ED hot
path at Ns = 14 (2x7 ladder, n_up = n_dn = 7, D = 11,778,624, m = 30), the
complex64 Krylov form (float64 Lanczos scalars) against the complex128 form,
plus the H.v bandwidth of the apply kernel against the HBM peak.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  With N > 1 (launched by torch.distributed.run)
every rank propagates its own copy of the workload (independent replicas, no
collective on the data path); value = (max-rank time) / (N * K).

The reference arm (--impl reference) times the float64 CPU oracle on the host
cores: every timed step is one whole oracle midpoint step of the same
workload (cpu_full_step()), the warm-up steps a bounded sample (cpu_warmup()).
"""
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "ladder2x7"
METRIC = "ms per midpoint time step (Ns=14 ladder, complex64 Krylov vectors, float64 Lanczos scalars)"
UNIT = "ms/step"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline timing (for profiler launch lists)")
    ap.add_argument("--random-start", action="store_true",
                    help="start from a seeded random state instead of the ground state")
    ap.add_argument("--no-spectral", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true")
    ap.add_argument("--no-ns16", action="store_true", help="skip the Ns=16 torus")
    ap.add_argument("--no-cfet4", action="store_true")
    ap.add_argument("--m", type=int, default=0,
                    help="Krylov dimension override for profiling runs (0: the workload's)")
    ap.add_argument("--apply-config", type=int, default=None,
                    help="pin the H v kernel configuration (default: autotuned)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the ring and torus workloads")
    ap.add_argument("--small-steps", type=int, default=20)
    ap.add_argument("--spectral-steps", type=int, default=2)
    ap.add_argument("--apply-only", choices=["c64", "c128"], default=None,
                    help="run 4 plain applies at the bench size and exit (profiler target)")
    ap.add_argument("--apply-workload", default=WORKLOAD,
                    help="workload of --apply-only (default: the bench's ladder)")
    ap.add_argument("--spectral-only", action="store_true",
                    help="run one small spectral batch (3x4 torus, 48 c/c+ vectors + psi, "
                         "m=4, 2 steps) and exit (profiler target of the overlap and "
                         "fermion-operator kernels)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; each sample
    keeps the host time it arrived at, so that summary() can keep the
    samples of one timed window."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock, max clock and active reasons of the samples that
        arrived between host times t0 and t1 (plus one sampling interval);
        all samples if that window holds none."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if t0 is not None and t1 is not None:
            win = [x for x in lines if t0 <= x[0] <= t1 + 0.05]
            lines = win or lines
        window = "timed region" if lines is not self.lines else "whole sampler run"
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_ms(t_ms, ws, device="cpu"):
    """Wall time of the whole job: the maximum over ranks of each rank's
    timed region (every rank runs an independent replica)."""
    if ws <= 1:
        return float(t_ms)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(t_ms, ws, steps):
    """ms per propagated midpoint step over the whole job: N replicas of K
    steps each finish in the max-over-ranks time."""
    return t_ms / (ws * steps)


def cpu_full_step(w, lat, psi=None, t=None):
    """One whole midpoint step of the oracle (float64: H(t_mid) as the scipy
    sparse Kronecker operator, m Lanczos iterations with NumPy BLAS-1, the
    m x m exponential and the combination, <d> and |psi|^2), as it stands,
    from a seeded state inside the pulse.  Returns (ms, psi after the step,
    t after the step, sample description)."""
    import oracle
    if psi is None:
        D = oracle.sector_dims(lat["Ns"], w["n_up"], w["n_dn"])[2]
        psi = np.asarray(__import__("synth").complex_normal(D, 0))
    if t is None:
        t = w["pulse_params"]["t0"] - 1.0
    t0 = time.perf_counter()
    r = oracle.propagate(lat, w["n_up"], w["n_dn"], w["U"], psi, w["pulse_params"], w["dt"],
                         1, w["m"], t_start=t, form="kron")
    ms = (time.perf_counter() - t0) * 1e3
    return ms, r["psi"], t + w["dt"], (f"one full midpoint step of the oracle (H(t_mid), "
                                       f"{w['m']} Lanczos iterations, exponential, combination, "
                                       f"<d>, |psi|^2), measured, not extrapolated")


def cpu_warmup(w, lat):
    """An untimed bounded sample: H(t_mid) and one product H v."""
    import oracle
    from oracle.krylov import make_H
    D = oracle.sector_dims(lat["Ns"], w["n_up"], w["n_dn"])[2]
    H = make_H(lat, w["n_up"], w["n_dn"], w["U"], oracle.pulse_A(9.01, w["pulse_params"]), "kron")
    H @ np.asarray(__import__("synth").complex_normal(D, 1))


def small_oracle_steps():
    """The oracle's ms per midpoint step on the ring (complex128, m=12, 20
    steps) and on the 3x4 torus (m=20, 2 steps), both from a seeded state
    inside the pulse: bounded samples of those trajectories, beside the GPU
    numbers of the same workloads."""
    import oracle
    import synth
    out = {}
    for name, steps in (("ring8", 20), ("torus3x4", 2)):
        w = synth.workload(name)
        lat = synth.lattice_from_name(w["lattice"])
        D = oracle.sector_dims(lat["Ns"], w["n_up"], w["n_dn"])[2]
        psi = synth.complex_normal(D, 0)
        t0 = time.perf_counter()
        oracle.propagate(lat, w["n_up"], w["n_dn"], w["U"], psi, w["pulse_params"], w["dt"],
                         steps, w["m"], t_start=w["pulse_params"]["t0"] - 1.0)
        out[name] = {"ms_per_step": (time.perf_counter() - t0) * 1e3 / steps, "steps": steps,
                     "m": w["m"], "kind": "oracle (float64, NumPy/SciPy)"}
    return out


def spectral_bench(ed, torch, synth, lat, w, pulse, h, psi64, stream, barrier, steps):
    m_spec = 20
    t0 = pulse["t0"] - 1.0
    gl = np.zeros(0)
    # warm-up call builds the batch (sectors, maps, 100 GB of Krylov storage)
    ed.ed_spectral_propagate(h.ctx, psi64, ed.ED_C64, pulse, w["dt"], 1, m_spec, 14,
                             stream=stream)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ed.ed_spectral_propagate(h.ctx, psi64, ed.ED_C64, pulse, w["dt"], steps, m_spec, 14,
                             stream=stream)
    e1.record(stream)
    barrier()
    batched = e0.elapsed_time(e1) / steps
    # one complex128 propagation of a c_i,up psi vector (sector (6,7)), per step
    hs = ed.Hubbard(lat, w["n_up"] - 1, w["n_dn"], w["U"])
    phi = torch.from_numpy(synth.complex_normal(hs.D, 5)).cuda()
    ed.ed_propagate(hs.ctx, phi, ed.ED_C128, pulse, t0, w["dt"], 1, m_spec, stream=stream)
    barrier()
    e0.record(stream)
    ed.ed_propagate(hs.ctx, phi, ed.ED_C128, pulse, t0, w["dt"], 2, m_spec, stream=stream)
    e1.record(stream)
    barrier()
    one64 = e0.elapsed_time(e1) / 2
    hs.close()
    del gl
    return {"workload": "Ns=14 ladder spectral batch: 56 c/c+ vectors of dim 10,306,296 + "
                        "psi, m=20, dt=0.02",
            "ms_per_step_batched_c64": batched, "steps": steps,
            "ms_per_step_sequential_c128": 56 * one64,
            "ms_per_vector_step_c128": one64,
            "speedup_batched_c64_over_sequential_c128": 56 * one64 / batched,
            "note": "sequential = 56 x one measured complex128 propagation step of "
                    "a vector of the same dimension"}


def kernel_sources_sha256():
    """sha256 over every file of csrc/ (sorted by name) and include/ed.h."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_13498_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "ed.h"), "rb").read())
    return h.hexdigest()


def profiled_traffic(apply_config):
    """DRAM bytes per Lanczos-pass apply from the committed ncu summary, or
    None when the kernel sources or the configuration differ from the
    profiled ones (the counters no longer describe this kernel)."""
    import re
    path = os.path.join(ROOT, "profiles", "apply_ladder2x7_c64_lanczos_dram.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    want = re.search(r"kernel_sources_sha256: ([0-9a-f]+)", txt)
    val = re.search(r"traffic_bytes_per_launch: (\d+)", txt)
    cfg = re.search(r"apply configuration (\d+)", txt)
    if not (want and val and cfg) or int(cfg.group(1)) != apply_config:
        return None
    return int(val.group(1)) if kernel_sources_sha256() == want.group(1) else None


def adaptive_bench(ed, torch, h, psi32, pulse, t_start, dt, m, stream, barrier, steps):
    """ms per step of the ladder workload with the adaptive exit at two
    tolerances (complex64), with the Krylov dimensions the steps used."""
    res = {}
    for tol in (1e-6, 1e-8):
        ed.ed_set_krylov_tol(h.ctx, tol)
        psi = psi32.clone()
        ed.ed_propagate(h.ctx, psi, ed.ED_C64, pulse, t_start - 2 * dt, dt, 2, m, stream=stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ed.ed_propagate(h.ctx, psi, ed.ED_C64, pulse, t_start, dt, steps, m,
                              stream=stream)
        e1.record(stream)
        barrier()
        me = out["m_eff"]
        res[f"tol={tol:g}"] = {"ms_per_step_c64": e0.elapsed_time(e1) / steps,
                               "m_eff_mean": float(np.mean(me)), "m_eff_min": int(me.min()),
                               "m_eff_max": int(me.max()), "steps": steps}
    ed.ed_set_krylov_tol(h.ctx, 0.0)
    res["note"] = ("m = 30 is the maximum; one Lanczos pass past the exit is computed "
                   "while the check runs")
    return res


def ns16_bench(ed, torch, synth, stream, barrier, steps, peak):
    """Ns=16 4x4 torus at half filling, (8,8), D = 165,636,900 (1.3 GB per
    complex64 vector): ms per midpoint step (complex64, m = 30, fixed and
    with the adaptive exit at 1e-8) from a seeded random state inside the
    pulse, and plain H v in both precisions."""
    w = synth.workload("torus4x4")
    lat = synth.lattice_from_name(w["lattice"])
    p, dt, m = w["pulse_params"], w["dt"], w["m"]
    h = ed.Hubbard(lat, w["n_up"], w["n_dn"], w["U"])
    D = h.D
    gen = torch.Generator(device="cuda").manual_seed(0)
    psi = torch.randn(D, dtype=torch.complex64, device="cuda", generator=gen)
    psi /= torch.linalg.vector_norm(psi)
    t_start = p["t0"] - 1.0
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {"workload": "Ns=16 4x4 torus, (8,8), D=165,636,900, U=8, m=30, dt=0.02, "
                       "pulse A0=0.5 Omega=8 sigma=2 t0=5 along (1,1)", "steps": steps}
    for tol in (0.0, 1e-8):
        ed.ed_set_krylov_tol(h.ctx, tol)
        ed.ed_propagate(h.ctx, psi, ed.ED_C64, p, t_start - dt, dt, 1, m, stream=stream)
        barrier()
        e0, e1 = ev(), ev()
        e0.record(stream)
        out = ed.ed_propagate(h.ctx, psi, ed.ED_C64, p, t_start, dt, steps, m, stream=stream)
        e1.record(stream)
        barrier()
        key = "fixed_m30" if tol == 0.0 else "adaptive_1e-8"
        res[key] = {"ms_per_step_c64": e0.elapsed_time(e1) / steps,
                    "m_eff_mean": float(np.mean(out["m_eff"]))}
    ed.ed_set_krylov_tol(h.ctx, 0.0)
    ed.ed_set_field(h.ctx, pulse_field(p, t_start))
    for name, tt, code, esz, n in (("c64", torch.complex64, ed.ED_C64, 8, 10),
                                   ("c128", torch.complex128, ed.ED_C128, 16, 3)):
        v = psi.to(tt)
        wv = torch.empty_like(v)
        ed.ed_apply_H(h.ctx, v, wv, code, stream=stream)
        barrier()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(n):
            ed.ed_apply_H(h.ctx, v, wv, code, stream=stream)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / n
        gbs = 2 * D * esz / (ms * 1e-3) / 1e9
        res[f"hv_{name}"] = {"ms": ms, "GBs": gbs, "frac_of_peak": gbs / peak}
        del v, wv
    res["apply_config_c64_step"] = ed.ed_get_apply_config(h.ctx)[0]
    h.close()
    return res


def cfet4_bench(ed, torch, h, psi32, pulse, t_start, m, stream, barrier):
    """Accuracy per cost on the ladder workload inside the pulse (complex64,
    m = 30): the midpoint rule at dt = 0.02 against CFET4 at dt = 0.08 over
    the same time window T = 0.32, both compared with CFET4 at dt = 0.01
    (the reference); time per unit of physical time."""
    T = 0.32
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def run(scheme, dt):
        ed.ed_set_integrator(h.ctx, scheme)
        psi = psi32.clone()
        n = int(round(T / dt))
        barrier()
        e0, e1 = ev(), ev()
        e0.record(stream)
        ed.ed_propagate(h.ctx, psi, ed.ED_C64, pulse, t_start, dt, n, m, stream=stream)
        e1.record(stream)
        barrier()
        return psi, e0.elapsed_time(e1)

    run("cfet4", 0.08)          # warm-up (engine setup, graph capture)
    ref, _ = run("cfet4", 0.01)
    res = {"window": f"T = {T} from t = {t_start}", "reference": "CFET4, dt = 0.01"}
    for scheme, dt in (("midpoint", 0.02), ("cfet4", 0.08), ("cfet4", 0.04)):
        run(scheme, dt)         # engine for this step count
        psi, ms = run(scheme, dt)
        err = float(torch.linalg.vector_norm(psi.to(torch.complex128) - ref.to(torch.complex128)))
        res[f"{scheme} dt={dt}"] = {"ms_per_unit_time": ms / T, "state_error": err}
    ed.ed_set_integrator(h.ctx, "midpoint")
    return res


def pulse_field(p, t):
    """A(t) = A0 exp(-(t - t0)^2 / (2 sigma^2)) sin(Omega (t - t0)) dir."""
    s = t - p["t0"]
    a = p["A0"] * math.exp(-s * s / (2.0 * p["sigma"] ** 2)) * math.sin(p["omega"] * s)
    return [a * c for c in p["dir"]]


def smaller_workloads_bench(ed, torch, synth, stream, barrier, steps):
    """The Ns=8 ring (complex128, m=12) and the 3x4 torus (both precisions,
    m=20): ms per midpoint step from the ground state at t=0; 100 applies of
    H on the seed-0 vector at A=0 and at A(dt/2); the torus spectral batch
    (48 c/c+ vectors + psi, complex64, m=20).  These vectors (<= 14 MB) stay
    in L2: no flush, no HBM fraction claimed."""
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    tdt = {"c128": (ed.ED_C128, torch.complex128), "c64": (ed.ED_C64, torch.complex64)}
    for name in ("ring8", "torus3x4"):
        w = synth.workload(name)
        lat = synth.lattice_from_name(w["lattice"])
        p, dt, m = w["pulse_params"], w["dt"], w["m"]
        h = ed.Hubbard(lat, w["n_up"], w["n_dn"], w["U"])
        g = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
        E0, _ = ed.ed_ground_state(h.ctx, g, tol=1e-10, max_iter=3000)
        res = {"D": h.D, "m": m, "dt": dt, "E0": E0}
        for name_dt in w["dtypes"]:
            code, tt = tdt[name_dt]
            psi = g.clone().to(tt)
            ed.ed_propagate(h.ctx, psi, code, p, 0.0, dt, 3, m, stream=stream)
            barrier()
            e0, e1 = ev(), ev()
            e0.record(stream)
            ed.ed_propagate(h.ctx, psi, code, p, 3 * dt, dt, steps, m, stream=stream)
            e1.record(stream)
            barrier()
            res[f"ms_per_step_{name_dt}"] = e0.elapsed_time(e1) / steps
        res["steps"] = steps
        if name == "torus3x4":
            v0 = synth.complex_normal(h.D, 0)
            hv = {}
            for label, A in (("A=0", [0.0, 0.0, 0.0]), ("A(dt/2)", pulse_field(p, dt / 2))):
                ed.ed_set_field(h.ctx, A)
                for name_dt in ("c128", "c64"):
                    code, tt = tdt[name_dt]
                    v = torch.from_numpy(v0).to(tt).cuda()
                    wv = torch.zeros_like(v)
                    for _ in range(3):
                        ed.ed_apply_H(h.ctx, v, wv, code, stream=stream)
                    barrier()
                    e0, e1 = ev(), ev()
                    e0.record(stream)
                    for _ in range(100):
                        ed.ed_apply_H(h.ctx, v, wv, code, stream=stream)
                    e1.record(stream)
                    barrier()
                    ms = e0.elapsed_time(e1) / 100
                    esz = 16 if name_dt == "c128" else 8
                    hv[f"{label} {name_dt}"] = {"us": ms * 1e3,
                                                "GBs": 2 * h.D * esz / (ms * 1e-3) / 1e9}
            res["hv_100_applies_seed0"] = hv
            # spectral batch of the torus from the same ground state
            ws = synth.workload("torus3x4_spectral")
            ed.ed_spectral_propagate(h.ctx, g, ed.ED_C64, p, ws["dt"], 1, ws["m"], 12,
                                     stream=stream)
            barrier()
            e0, e1 = ev(), ev()
            e0.record(stream)
            ed.ed_spectral_propagate(h.ctx, g, ed.ED_C64, p, ws["dt"], steps, ws["m"], 12,
                                     stream=stream)
            e1.record(stream)
            barrier()
            bms = e0.elapsed_time(e1) / steps
            # A(nu, t_ref) at t_ref = 1.0 (Eq. (15) and Eq. (37)):
            # psi to t_ref, the batch from t_ref, the broadened transform
            t_ref, n_tr = 1.0, 2 * steps
            x = g.clone()
            barrier()
            e0, e1 = ev(), ev()
            e0.record(stream)
            ed.ed_propagate(h.ctx, x, ed.ED_C128, p, 0.0, ws["dt"], int(round(t_ref / ws["dt"])),
                            ws["m"], stream=stream)
            Gl, Gg = ed.ed_spectral_propagate_at(h.ctx, x, t_ref, ed.ED_C64, p, ws["dt"], n_tr,
                                                 ws["m"], 12, stream=stream)
            nu = np.linspace(-12.0, 12.0, 241)
            Anu = (ed.ed_spectral_function(Gl, ws["dt"], 0.2, nu) +
                   ed.ed_spectral_function(Gg, ws["dt"], 0.2, nu))
            e1.record(stream)
            barrier()
            out["torus3x4_A_nu_tref"] = {
                "workload": f"A(nu, t_ref = {t_ref}) of the 3x4 torus: psi propagated to t_ref "
                            f"(complex128, m=20), {n_tr} batch steps (complex64), transform on "
                            f"{len(nu)} frequencies, eps = 0.2",
                "ms_total": e0.elapsed_time(e1), "A_site_avg_max": float(Anu.mean(axis=(1, 2)).max())}
            out["torus3x4_spectral"] = {
                "workload": "Ns=12 3x4 torus spectral batch: 48 c/c+ vectors of dim 731,808 "
                            "+ psi, complex64, m=20, dt=0.02",
                "ms_per_step_batched_c64": bms, "ms_per_vector_step": bms / 49,
                "steps": steps}
        h.close()
        out[name] = res
    return out


def bench_config(t_start, m, ws):
    """The workload description both arms print (identical dicts)."""
    return {"workload": "Ns=14 2x7 ladder (periodic legs, open rungs), n_up=n_dn=7, "
                        "D=11,778,624, U=8, m=30, dt=0.02, pulse A0=0.5 Omega=8 "
                        "sigma=2 t0=10 along the legs",
            "t_start": t_start, "m": m, "parallelism": f"replicas x{ws}",
            "l2": "no flush: per-step working set 2.9 GB (31 Krylov vectors of "
                  "94 MB) > 129 MB L2"}


def reference_arm(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import synth
    w = synth.workload(WORKLOAD)
    lat = synth.lattice_from_name(w["lattice"])
    for _ in range(args.warmup):
        cpu_warmup(w, lat)
    per = []
    psi, t = None, None
    desc = ""
    # whole oracle steps, measured one by one, until the time budget is used
    # (at least one): one step takes about 20 s on 16 host cores, so K = 20
    # full steps would hold the GPUs for minutes
    budget_s = 150.0
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        ms, psi, t, desc = cpu_full_step(w, lat, psi, t)
        per.append(ms)
        if time.perf_counter() - t0 >= budget_s:
            break
    val = float(np.mean(per))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": len(per), "steps_requested": args.steps,
            "warmup": args.warmup,
            "ms_per_step": val, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w["pulse_params"]["t0"] - 1.0, w["m"], 1),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc + f"; {len(per)} consecutive steps measured "
                                              f"({args.steps} requested; whole steps until "
                                              f"{budget_s:.0f} s were used), "
                                              f"warm-up: {args.warmup} x (H(t_mid), one H v)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import synth
    from paper_2005_13498_gb300 import build as _b
    _b.build()
    from paper_2005_13498_gb300 import ed

    w = synth.workload(WORKLOAD)
    lat = synth.lattice_from_name(w["lattice"])
    pulse = w["pulse_params"]
    dt, m = w["dt"], w["m"]
    if args.m:            # profiling a smaller Krylov space (not the headline)
        m = args.m
    if args.apply_config is not None:
        ed.ed_set_apply_config(args.apply_config)
    if args.apply_only:
        if args.apply_workload != WORKLOAD:
            w = synth.workload(args.apply_workload)
            lat = synth.lattice_from_name(w["lattice"])
        h = ed.Hubbard(lat, w["n_up"], w["n_dn"], w["U"])
        ed.ed_set_field(h.ctx, [0.3, 0.0, 0.0])
        tt, code = ((torch.complex64, ed.ED_C64) if args.apply_only == "c64"
                    else (torch.complex128, ed.ED_C128))
        v = torch.from_numpy(synth.complex_normal(h.D, 0)).to(tt).cuda()
        wv = torch.zeros_like(v)
        for _ in range(4):
            ed.ed_apply_H(h.ctx, v, wv, code)
        torch.cuda.synchronize()
        print(json.dumps({"apply_only": args.apply_only, "D": h.D,
                          "config": ed.ed_get_apply_config(h.ctx)[1]}))
        h.close()
        return
    if args.spectral_only:
        ws_ = synth.workload("torus3x4_spectral")
        lat_ = synth.lattice_from_name(ws_["lattice"])
        h = ed.Hubbard(lat_, ws_["n_up"], ws_["n_dn"], ws_["U"])
        psi = torch.from_numpy(synth.complex_normal(h.D, 0)).cuda()
        gl, gg = ed.ed_spectral_propagate(h.ctx, psi, ed.ED_C64, ws_["pulse_params"],
                                          ws_["dt"], 2, 4, 12)
        torch.cuda.synchronize()
        print(json.dumps({"spectral_only": "torus3x4", "D": h.D,
                          "G_less_00": [float(gl[0, 0, 0].real), float(gl[0, 0, 0].imag)]}))
        h.close()
        return
    t_start = pulse["t0"] - 1.0        # inside the pulse: full Krylov dimension
    h = ed.Hubbard(lat, w["n_up"], w["n_dn"], w["U"])
    D = h.D
    stream = torch.cuda.current_stream()

    # S0 (one-off, untimed): ground state in float64
    g = torch.zeros(D, dtype=torch.complex128, device="cuda")
    if args.random_start:
        g.copy_(torch.from_numpy(synth.complex_normal(D, 0)))
        E0, resid = None, None
    else:
        E0, resid = ed.ed_ground_state(h.ctx, g, tol=1e-10, max_iter=3000)
    psi64 = g.clone()
    psi32 = g.to(torch.complex64)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- headline
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:      # running before the timed region starts
        ed.ed_propagate(h.ctx, psi32, ed.ED_C64, pulse, t_start - args.warmup * dt, dt,
                        args.warmup, m, stream=stream)
        psi_t0 = psi32.clone()          # the state at t_start, for the later legs
        barrier()
        time.sleep(0.3)
        h0 = time.time()
        e0.record(stream)
        out = ed.ed_propagate(h.ctx, psi32, ed.ED_C64, pulse, t_start, dt, args.steps, m,
                              stream=stream)
        e1.record(stream)
        barrier()
        h1 = time.time()
    t_ms = job_time_ms(e0.elapsed_time(e1), ws, device="cuda")
    value = job_value(t_ms, ws, args.steps)
    ms_step = t_ms / args.steps
    m_eff = out["m_eff"]
    # kernels per step: m applies (two kernels each for the split apply),
    # m - 1 updates, expm, combine; plus the observation launch and the two
    # column permutations (into the hop order of the down-spin tables and back)
    acfg = ed.ed_get_apply_config(h.ctx)[0]
    ainfo = ed.ed_apply_config_info(acfg)
    gpu_launches = 3 + args.steps * ((2 + ainfo["split"]) * m + 1)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": bench_config(t_start, m, ws), "m_eff_min": int(m_eff.min()),
            "clocks": clk.summary(h0, h1), "gpu_launches": gpu_launches,
            "apply_kernel": dict(ainfo, config=acfg),
            "ground_state": {"E0": E0, "residual": resid}}

    if not args.no_extras:
        peak, peak_kind = measured_peaks()
        # on-chip ceilings (L2 and shared-memory read rates, FMA rates) that
        # bound the apply when DRAM does not
        from paper_2005_13498_gb300 import probes
        line["ceilings"] = probes.ed_probe_ceilings()
        # per-kernel device time (event pair around every launch, same K steps)
        prof = ed.ed_propagate(h.ctx, psi32, ed.ED_C64, pulse, t_start, dt, args.steps, m,
                               profile=True, stream=stream)
        km, kl = prof["kernel_ms"], prof["kernel_launches"]
        names = ed.KERNEL_KIND_NAMES
        kern = {names[i]: {"ms_total": float(km[i]), "launches": int(kl[i]),
                           "ms_per_launch": float(km[i] / kl[i]) if kl[i] else None}
                for i in range(6) if kl[i]}
        tot = sum(float(km[i]) for i in range(6))
        for k in kern:
            kern[k]["share"] = kern[k]["ms_total"] / tot
        line["kernels"] = kern
        # dominant kernel: the Lanczos apply (one kernel, or column pass + row
        # pass for the split configuration, timed together); algorithmic bytes
        # per launch averaged over j = 1..m: read x_j (+ x_{j-1} for j >= 2),
        # write w.
        s = 8
        bytes_apply = (2 + 3 * (m - 1)) / m * D * s
        a_ms = kern["apply"]["ms_per_launch"]
        achieved = bytes_apply / (a_ms * 1e-3) / 1e9
        traffic = profiled_traffic(acfg)
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak,
                            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                            "traffic_note": "ncu dram read + write of one j >= 2 pass "
                                            "(profiles/apply_ladder2x7_c64_lanczos_dram.md); "
                                            "null if the kernel changed since",
                            "kernel": ("k_apply_up + k_apply (split" if ainfo["split"]
                                       else "k_apply (one kernel") +
                                      ": w = s_j H x_j - beta s x_{j-1}, <v_j,w>)",
                            "algorithmic_bytes_per_launch": bytes_apply,
                            "peak_kind": peak_kind + " (burst copy)"}
        # H.v bandwidth: 100 back-to-back plain applies (read v, write w)
        ed.ed_set_field(h.ctx, [float(synth.PULSES[WORKLOAD]["A0"]), 0.0, 0.0])
        v = torch.from_numpy(synth.complex_normal(D, 0)).to(torch.complex64).cuda()
        wv = torch.zeros_like(v)
        for _ in range(3):
            ed.ed_apply_H(h.ctx, v, wv, ed.ED_C64, stream=stream)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(100):
            ed.ed_apply_H(h.ctx, v, wv, ed.ED_C64, stream=stream)
        a1.record(stream)
        barrier()
        hv_ms = a0.elapsed_time(a1) / 100
        line["hv"] = {"GBs": 2 * D * 8 / (hv_ms * 1e-3) / 1e9, "ms": hv_ms,
                      "frac_of_peak": 2 * D * 8 / (hv_ms * 1e-3) / 1e9 / peak,
                      "note": "plain apply, 100 launches, bytes = 2 D 8 (complex64)"}
        v64 = v.to(torch.complex128)
        w64 = torch.zeros_like(v64)
        ed.ed_apply_H(h.ctx, v64, w64, ed.ED_C128, stream=stream)
        barrier()
        a0.record(stream)
        for _ in range(10):
            ed.ed_apply_H(h.ctx, v64, w64, ed.ED_C128, stream=stream)
        a1.record(stream)
        barrier()
        hv64 = a0.elapsed_time(a1) / 10
        line["hv_c128"] = {"GBs": 2 * D * 16 / (hv64 * 1e-3) / 1e9, "ms": hv64,
                           "config": ed.ed_get_apply_config(h.ctx)[1]}
        # float64 propagator on the same workload
        ed.ed_propagate(h.ctx, psi64, ed.ED_C128, pulse, t_start - dt, dt, 1, m, stream=stream)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ed.ed_propagate(h.ctx, psi64, ed.ED_C128, pulse, t_start, dt, args.fp64_steps, m,
                        stream=stream)
        f1.record(stream)
        barrier()
        fp64_ms = f0.elapsed_time(f1) / args.fp64_steps
        line["fp64"] = {"ms_per_step": fp64_ms, "steps": args.fp64_steps,
                        "speedup_c64_over_c128": fp64_ms / ms_step,
                        "apply_config": ed.ed_get_apply_config(h.ctx)[0]}
        # spectral batch (Ns=14 ladder): c and c^+ on every site and spin of
        # the state, 56 vectors of 3003x3432 / 3432x3003 plus psi, m=20,
        # complex64, one batched launch per kernel; against 56 sequential
        # complex128 propagations (one measured, times 56)
        if not args.no_spectral:
            line["spectral"] = spectral_bench(ed, torch, synth, lat, w, pulse, h, psi64,
                                              stream, barrier, args.spectral_steps)
        # adaptive Krylov dimension (a-posteriori exit of Algorithm 6, m = 30
        # as the maximum) on the same ladder workload: 20 steps from the
        # state at t_start, whatever --steps is
        if not args.no_adaptive:
            line["adaptive"] = adaptive_bench(ed, torch, h, psi_t0, pulse, t_start, dt, m,
                                              stream, barrier, 20)
        # fourth-order commutator-free integrator: accuracy per cost, from
        # the state at t_start
        if not args.no_cfet4:
            line["cfet4"] = cfet4_bench(ed, torch, h, psi_t0, pulse, t_start, m, stream,
                                        barrier)
        # Ns = 16 at half filling (beyond the paper's CSR memory limit)
        if not args.no_ns16:
            line["ns16"] = ns16_bench(ed, torch, synth, stream, barrier, 2, peak)
        # the ring and torus workloads (step times, H v on the seed-0 vector,
        # the torus spectral batch)
        if not args.no_small:
            line.update(smaller_workloads_bench(ed, torch, synth, stream, barrier,
                                                args.small_steps))
        # end to end through the C ABI with pinned host buffers: every step
        # copies psi in, propagates one step, copies psi and <d> out
        hostpsi = psi32.cpu().pin_memory()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ed.ed_propagate(h.ctx, hostpsi, ed.ED_C64, pulse, t_start + k * dt, dt, 1, m,
                            stream=stream)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        line["e2e"] = {"value": e2e_ms / ws, "unit": UNIT, "h2d_bytes_per_step": D * 8,
                       "d2h_bytes_per_step": D * 8 + 2 * 8 * 2,
                       "note": "one ed_propagate call per step on a pinned host buffer"}
        # CPU oracle on this host (rank 0, N = 1 only)
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            cms, _, _, desc = cpu_full_step(w, lat)
            cores = (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                     else os.cpu_count())
            line["cpu_baseline"] = {"value": cms, "unit": UNIT, "cores": cores,
                                    "kind": "oracle", "sample": desc}
            if not args.no_small:
                line["cpu_baseline_small"] = small_oracle_steps()
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
