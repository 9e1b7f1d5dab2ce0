"""Benchmark: Keldysh G(t,t') steps per second on the L = 12 Hubbard-ring quench.

Workload (one GPU): the Hubbard ring L = 12, T = 1, PBC, half filling (6,6),
d = 853,776; ground state at U = 8, quench to U = 4; dt = 0.05, Krylov M = 20,
full reorthogonalisation, grid of 100 times, all 12 spin-up orbitals.
A step is one row of step (iii) of the four-step method at the last grid time
t_99 = 4.95: the c and c^dag maps of Phi(t_99) (24 columns in the N-1 and N+1
sectors, d = 731,808 each), 99 backward Krylov steps per column
(2 x 12 x 99 = 2376 G-steps) and the time-diagonal block G^<,>(t_99, t_99).
Set-up (sector tables, ground state of H_ini, Phi(t_k) for all k) is not timed.

Timed region: CUDA events on the library's launch stream, W >= 3 warm-up
steps, K timed steps, barrier + synchronize on both sides, max over ranks.
Every step streams its 2.9 GB Krylov basis and ~1.1 GB of other vectors, far
beyond the 129 MB L2, so no flush is needed between steps.

Under torchrun (N > 1) every rank runs the same kind of row on its own GPU
(rank r takes row 99 - r); there is no collective on the data path (weak
scaling).  `--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·ψ GB/s (frac. of HBM peak); G(t,t') steps/s, batched+adjoint vs plain GPU"
UNIT = "G(t,t') steps/s"


def shard_rows(n_t, world, rank):
    """Rows of step (iii) owned by a rank: round robin from the costliest."""
    return [k for k in range(n_t - 1, -1, -1) if (n_t - 1 - k) % world == rank]


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# Algorithmic bytes (read + write of complex FP64 vectors, 16 B per element)
# of each kernel class over one propagation step of B columns of dimension d
# with Krylov dimension M, full reorthogonalisation (one Gram-Schmidt pass).
def step_bytes(d, B, M, n_ov=0):
    v = 16.0 * d * B
    hpsi = sum(v * (2 + (1 if j > 0 else 0)) for j in range(M))           # read V_j (+V_{j-1}), write W
    dots = sum(v * (2 + (j + 1)) for j in range(M))                         # W, V_j, V_0..V_j
    upd = sum(v * (3 + (j + 1)) for j in range(M))                          # W, V_j, V_0..V_j, write V_{j+1}
    comb = v * (M + 1 + n_ov)
    return {"lanczos_hpsi": hpsi, "reorth_dots": dots, "update": upd, "combine": comb, "colnorm": v}


def step_flops(d, B, M, hops, int_dots=True):
    """FP64 operations (FMA = 2) per propagation step, by kernel class.  With
    the exact integer Gram-Schmidt dots (the default schedule) the dots
    kernel's only FP64 work is u = W - a_j v_j; its products run on the
    integer pipe."""
    e = float(d) * B
    return {"lanczos_hpsi": sum(e * (2 * hops + 17) for _ in range(M)),
            "reorth_dots": sum(e * (4 if int_dots else 4 + 8 * (j + 1)) for j in range(M)),
            "update": sum(e * (4 + 8 * (j + 1) + 4) for j in range(M)),
            "combine": e * 8 * (M + 1), "colnorm": e * 4}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    cfg = W.config_c2()
    n_t, dt, M = cfg["n_t"], cfg["dt"], cfg["M"]
    orbs = cfg["orbitals"]
    stream = torch.cuda.Stream()
    opts = kg.kg_opts_default(M=M, reorth=1, stream=stream.cuda_stream)
    t_setup = time.perf_counter()
    si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
    E0, res, gap = si.ground_state(opts)
    K = kg.Keldysh(si, sf, orbs, dt, n_t, opts)
    t_setup = time.perf_counter() - t_setup
    k_row = shard_rows(n_t, world, rank)[0]
    d_nb = sf.neighbour_dim(0, False)
    gsteps = 2 * len(orbs) * k_row  # (les, gtr) x orbitals x k backward steps

    for _ in range(args.warmup):
        K.row(k_row)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    gpu_index = local
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    n0 = kg.kg_launch_count()
    with ClockSampler(gpu_index) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps
        e0.record(stream)
        for _ in range(args.steps):
            K.row(k_row)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier()
    launches = kg.kg_launch_count() - n0
    t = e0.elapsed_time(e1) * 1e-3
    t_max = t
    total_gsteps = gsteps * args.steps
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        gg = torch.tensor([total_gsteps], dtype=torch.float64, device="cuda")
        dist.all_reduce(gg, op=dist.ReduceOp.SUM)
        total_gsteps = float(gg.item())
    value = total_gsteps / t_max

    # ---- end to end through the C ABI with host buffers: Phi(t_k) from pinned
    # host memory in, the G(t_k, t_k) block back to host memory, every step.
    phi_host = torch.empty(sf.dim, dtype=torch.complex128).pin_memory()
    phi_host.numpy()[:] = K.get_phi(k_row)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ke = args.steps
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(ke):
        K.set_phi(k_row, phi_host.numpy())
        K.row(k_row)
    e3.record(stream)
    torch.cuda.synchronize()
    t_e2e = e2.elapsed_time(e3) * 1e-3
    e2e = {"value": gsteps * ke / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 16 * sf.dim,
           "d2h_bytes_per_step": 2 * 16 * len(orbs) ** 2}

    # ---- roofline: per-kernel event timing of one profiled row
    peaks, peak_kind = read_peaks()
    fp64 = kg.kg_probe_fp64(stream)
    k_prof = min(k_row, 10)
    kg.kg_profile_start()
    K.row(k_prof)
    prof = kg.kg_profile_stop()
    n_prof_steps = 2 * k_prof  # propagation steps (each of 12 columns) in the profiled row
    # mean allowed ring hops per state of the (5,6) column sector: 2L bonds x
    # P(site occupied, neighbour empty) summed over both spins
    L_, nu_, nd_ = 12, 5, 6
    hops = 2.0 * L_ * (nu_ * (L_ - nu_) + nd_ * (L_ - nd_)) / (L_ * (L_ - 1))
    by = step_bytes(d_nb, len(orbs), M)
    fl = step_flops(d_nb, len(orbs), M, hops)
    kernels = {}
    tot_ms = sum(ms for _, ms in prof.values()) or 1.0
    for name, (n, ms) in prof.items():
        ent = {"launches": n, "ms": round(ms, 3), "share": round(ms / tot_ms, 4)}
        if name in by:
            ent["gbs"] = round(by[name] * n_prof_steps / (ms * 1e-3) / 1e9, 1)
            ent["tflops_fp64"] = round(fl[name] * n_prof_steps / (ms * 1e-3) / 1e12, 3)
        kernels[name] = ent
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    hbm_frac = dk.get("gbs", 0.0) / peaks["hbm_gbs"]
    fp_frac = dk.get("tflops_fp64", 0.0) / fp64
    # DRAM traffic of the dominant kernel: the traffic/algorithmic ratio of an
    # ncu capture (profiles/traffic.json) times this launch's algorithmic bytes,
    # null once the kernel sources differ from the captured ones.
    traffic = None
    tj = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tj) and dom in by:
        rec = json.load(open(tj)).get(dom)
        if rec and rec.get("source_hash") == source_hash(rec.get("sources", [])):
            per_launch = by[dom] * n_prof_steps / max(1, prof[dom][0])
            traffic = round(rec["ratio"] * per_launch)
    if hbm_frac >= fp_frac:
        roof = {"bound": "hbm", "achieved": dk.get("gbs"), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(hbm_frac, 4), "traffic": traffic, "kernel": dom,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": dk.get("tflops_fp64"), "peak": round(fp64, 3), "unit": "TFLOP/s",
                "frac": round(fp_frac, 4), "traffic": traffic, "kernel": dom,
                "peak_source": "FP64 FMA throughput measured live by kg_probe_fp64"}

    # ---- H*psi alone (the metric's first half), buffers rotated beyond L2
    nbuf = 12
    xs = [torch.randn(d_nb, dtype=torch.complex128, device="cuda") for _ in range(nbuf)]
    ys = [torch.empty_like(x) for x in xs]
    nb_sec = kg.Sector(W.with_sector(cfg["fin"], 5, 6))
    with torch.cuda.stream(stream):
        for i in range(nbuf):
            nb_sec.hpsi(xs[i], ys[i], stream)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        h0.record(stream)
        for _ in range(reps):
            for i in range(nbuf):
                nb_sec.hpsi(xs[i], ys[i], stream)
        h1.record(stream)
        torch.cuda.synchronize()
        # device time of each call (its kernels between CUDA events on the
        # launch stream), without the host's issue gaps between calls
        kg.kg_profile_start()
        for _ in range(reps):
            for i in range(nbuf):
                nb_sec.hpsi(xs[i], ys[i], stream)
        hprof = kg.kg_profile_stop()
    t_wall = h0.elapsed_time(h1) * 1e-3 / (reps * nbuf)
    n_h, ms_h = hprof.get("hpsi", (1, float("nan")))
    t_h = ms_h * 1e-3 / max(1, n_h)
    hpsi = {"d": d_nb, "us": round(t_h * 1e6, 2), "gbs": round(32.0 * d_nb / t_h / 1e9, 1),
            "frac_hbm": round(32.0 * d_nb / t_h / 1e9 / peaks["hbm_gbs"], 4),
            "us_back_to_back": round(t_wall * 1e6, 2),
            "algorithmic_bytes": 32 * d_nb, "l2": "12 rotating x/y pairs, 281 MB > L2",
            "timing": "device time per call from CUDA events around its kernels; us_back_to_back includes "
                      "the host's issue time between calls"}

    # ---- H*psi alone on a vector eleven times the L2 (the column sector of
    # the 16-site chain, d = 91,611,520, 1.47 GB)
    big = kg.Sector(W.with_sector(W.config_c3()["fin"], 6, 7))
    xb = torch.randn(big.dim, dtype=torch.complex128, device="cuda")
    yb = torch.empty_like(xb)
    with torch.cuda.stream(stream):
        big.hpsi(xb, yb, stream)
        torch.cuda.synchronize()
        kg.kg_profile_start()
        for _ in range(5):
            big.hpsi(xb, yb, stream)
        bprof = kg.kg_profile_stop()
    n_b, ms_b = bprof.get("hpsi", (1, float("nan")))
    t_b = ms_b * 1e-3 / max(1, n_b)
    hpsi["c3_column"] = {"d": big.dim, "us": round(t_b * 1e6, 1), "gbs": round(32.0 * big.dim / t_b / 1e9, 1),
                         "frac_hbm": round(32.0 * big.dim / t_b / 1e9 / peaks["hbm_gbs"], 4),
                         "algorithmic_bytes": 32 * big.dim}
    del xb, yb, big
    torch.cuda.empty_cache()

    # ---- CPU baseline: the oracle on the host cores, a bounded sample
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args.cpu_seconds)

    # ---- the batched and adjoint forms against the plain GPU path
    batched = adjoint = spectral = c2_full = c3_row = driven = None
    if rank == 0 and world == 1 and not args.no_extras:
        batched = batched_vs_plain(args.batch_instances, args.batch_steps, args.plain_steps)
        adjoint = adjoint_vs_fd()
        spectral = lanczos_spectral(si, opts)
        spectral["fine_grid"] = fine_grid_vs_plain(si, opts)
        spectral["fourier"] = fourier_transform(fp64)
        spectral["fig1"] = fig1_restarts()
        driven = driven_vs_quench(si, sf, opts)
        driven["four_time"] = four_time(si, sf, opts)
        driven["necpt"] = necpt_fig5(sizes=(4,), dtau=0.1)
        if not args.no_c2_full:
            c2_full = c2_full_grid(si, sf, opts)
    if rank == 0 and world == 1 and args.c3:
        c3_row = c3_rows(args.c3_nt)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": row_workload(k_row),
                       "global_batch_gsteps_per_step": gsteps * world, "columns": 2 * len(orbs),
                       "sector_dim": sf.dim, "column_dim": d_nb, "M": M, "reorth": 1,
                       "l2": "inputs larger than L2 (2.9 GB Krylov basis per step)",
                       "parallelism": "rows sharded over %d rank(s), no data-path collective" % world},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "kernels": kernels, "hpsi": hpsi,
            "fp64_tflops_measured": round(fp64, 3), "cpu_baseline": cpu, "clocks": clocks,
            "setup_s": round(t_setup, 2), "E0_ini": E0, "gs_resid": res,
            "batched": batched, "adjoint": adjoint, "spectral": spectral, "c2_full": c2_full, "c3_row": c3_row,
            "driven": driven,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def row_workload(k_row):
    return ("c2 Hubbard ring L=12 (6,6) d=853776, U=8 -> U=4 quench; Keldysh step (iii) row t_%d: 24 columns x "
            "%d G-steps (dt=0.05, M=20, full reorth) + G(t_k,t_k) block" % (k_row, k_row))


def c2_full_grid(si, sf, opts):
    """Time to solution of the whole c2 quench through the C ABI's one-shot
    call kg_green_keldysh: step (ii) (Phi on 100 times), step (iii) for every
    row (both kinds, 12 columns each, k backward G-steps in row k) and the
    step-(iv) Gram of 1,200 vectors per kind, results on the host.  The ground
    state of H_ini is the benchmark's own (already computed)."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c2()
    orbs, dt, n_t = cfg["orbitals"], cfg["dt"], cfg["n_t"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gl, Gg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, dt, n_t, opts)
    sec = time.perf_counter() - t0
    gsteps = (n_t - 1) + 2 * len(orbs) * n_t * (n_t - 1) // 2
    t = np.arange(n_t)
    sum_rule = float(np.max(np.abs(1j * (Gg[t, t] - Gl[t, t]) - np.eye(len(orbs))[None])))
    transl = float(max(np.max(np.abs(np.roll(np.roll(G, 1, 2), 1, 3) - G)) for G in (Gl, Gg)))
    return {"workload": "c2 quench, whole 100x100 grid, all 12x12 spin-up pairs, G^< and G^> (Phi steps, every row of "
                        "step (iii), 1200-vector Gram per kind) through kg_green_keldysh",
            "seconds": round(sec, 2), "gsteps": gsteps, "gsteps_per_s": round(gsteps / sec, 1),
            "max_sum_rule_dev": sum_rule, "max_translation_dev": transl}


# where the driven Keldysh calls sample the drive within an internal step h:
# the two Gauss-Legendre nodes t + (1/2 -+ sqrt(3)/6) h (include/krylovgf.h)
GAUSS2 = (0.5 - math.sqrt(3.0) / 6.0, 0.5 + math.sqrt(3.0) / 6.0)


def driven_vs_quench(si, sf, opts, n_t=11):
    """The c2 ring under a drive after the quench (every on-site energy
    oscillating, U of site 0 modulated): the whole n_t x n_t grid for all 12
    spin-up orbitals through kg_green_keldysh_td (fourth-order commutator-free
    steps, two Krylov exponentials of dt/2 per step) against the undriven
    quench through kg_green_keldysh on the same grid; then the order of the
    driven steps at full size: the grid at t = 0.4 for h = 0.2, 0.1, 0.05
    (self-convergence ratio |G_h - G_h/2| / |G_h/2 - G_h/4|, 16 for order 4)."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c2()
    orbs, dt = cfg["orbitals"], cfg["dt"]
    f = W.periodic_drive(12)
    dp = W.drive_samples(f, dt, n_t, 1, GAUSS2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gl, Gg = kg.kg_green_keldysh_td(si.handle, sf.handle, orbs, dt, n_t, dp, opts)
    sec_td = time.perf_counter() - t0
    t0 = time.perf_counter()
    Ql, Qg = kg.kg_green_keldysh(si.handle, sf.handle, orbs, dt, n_t, opts)
    sec_q = time.perf_counter() - t0
    gsteps = (n_t - 1) + 2 * len(orbs) * n_t * (n_t - 1) // 2
    t = np.arange(n_t)
    sum_rule = float(np.max(np.abs(1j * (Gg[t, t] - Gl[t, t]) - np.eye(len(orbs))[None])))
    # self-convergence in h on a 3-point grid (t = 0, 0.2, 0.4), two orbitals
    o2 = orbs[:2]
    errs, grids = [], []
    for n_sub in (1, 2, 4):
        o = kg.kg_opts_default(M=opts.M, reorth=opts.reorth, dt_internal=0.2 / n_sub)
        o.stream = opts.stream
        grids.append(kg.kg_green_keldysh_td(si.handle, sf.handle, o2, 0.2, 3,
                                            W.drive_samples(f, 0.2, 3, n_sub, GAUSS2), o))
    for a, b in zip(grids, grids[1:]):
        errs.append(float(max(np.max(np.abs(a[0] - b[0])), np.max(np.abs(a[1] - b[1])))))
    return {"workload": "c2 ring (6,6) d=853776 after the U=8 -> 4 quench with a drive (eps_i(t) = 0.7 sin(1.3 t + "
                        "phase), U_0(t) = 4 + 0.8 cos(2.1 t)); %dx%d grid, 12 spin-up orbitals, G^< and G^>, "
                        "dt=0.05, M=20" % (n_t, n_t),
            "seconds_driven": round(sec_td, 2), "seconds_quench": round(sec_q, 2), "gsteps": gsteps,
            "gsteps_per_s_driven": round(gsteps / sec_td, 1), "gsteps_per_s_quench": round(gsteps / sec_q, 1),
            "max_sum_rule_dev": sum_rule, "max_driven_minus_quench": float(np.max(np.abs(Gl - Ql))),
            "self_convergence": {"h": [0.2, 0.1, 0.05], "diffs": errs,
                                 "ratio": round(errs[0] / errs[1], 2) if errs[1] > 0 else None}}


def four_time(si, sf, opts, n_t=8):
    """A four-time correlation function of the c2 quench (the higher-order
    Green's functions of the paper's outlook): <0|c_0up(t1) c_1dn(t2)
    c^dag_1dn(t3) c^dag_0up(t4)|0> on an n_t^4 grid at dt = 0.05 through
    kg_green_four_time; the right and left two-time vector families of the
    (7,7) sector and their n_t^2 x n_t^2 overlap matrix."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    ops = [(0, 0, 0), (1, 1, 0), (1, 1, 1), (0, 0, 1)]
    dt = 0.05
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G = kg.kg_green_four_time(si.handle, sf.handle, ops, dt, n_t, opts)
    sec = time.perf_counter() - t0
    per_family = n_t * (2 * (n_t - 1) + n_t * (n_t - 1) // 2)
    gsteps = (n_t - 1) + 2 * per_family
    eq = np.array([G[k, k, k, k] for k in range(n_t)])
    return {"workload": "c2 ring after the U=8 -> 4 quench: <c_0up(t1) c_1dn(t2) c^dag_1dn(t3) c^dag_0up(t4)> "
                        "on a %d^4 grid, dt=0.05, M=20 (two families of %d vectors in the (7,7) sector, "
                        "d=627264)" % (n_t, n_t * n_t),
            "seconds": round(sec, 2), "gsteps": gsteps, "gsteps_per_s": round(gsteps / sec, 1),
            "equal_time_values": [round(float(v.real), 12) for v in eq],
            "max_equal_time_imag": float(np.max(np.abs(eq.imag)))}


def necpt_fig5(sizes=(4, 6), dt=0.05, t_max=5.0, beta=15.0, dtau=0.05, L_b=1000):
    """The NE-CPT of the paper's application (Fig. 5 model: impurity chain
    cluster of L_c sites, U = T = V = 1, field 0.2 on the impurity switched
    off at t = 0, coupled to a 1000-site bath) through kg_necpt_occupations:
    the initial moment m_1 = n_1up - n_1dn, the net moment of the first four
    sites and its decay on a coarse grid, per cluster size; seconds per call
    (cluster components on the GPU, contour LU on the device)."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    n_t = int(round(t_max / dt)) + 1
    n_tau = int(round(beta / dtau))
    out = {"workload": "NE-CPT, Fig. 5 model: L_b=%d bath, U=T=V=1, h=0.2 -> 0, dt=%g, t_max=%g, beta=%g, dtau=%g "
                       "(%d contour points)" % (L_b, dt, t_max, beta, dtau, 2 * n_t + n_tau + 1), "clusters": {}}
    for Lc in sizes:
        si = kg.Sector(W.siam_chain(Lc, 1.0, Lc // 2, Lc // 2, field=0.2))
        sf = kg.Sector(W.siam_chain(Lc, 1.0, Lc // 2, Lc // 2, field=0.0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = kg.kg_necpt_occupations(si, sf, L_b, 1.0, 1.0, dt, n_t, beta, n_tau)
        sec = time.perf_counter() - t0
        m = n[0] - n[1]
        step = int(round(1.0 / dt))
        out["clusters"][str(Lc)] = {
            "seconds": round(sec, 2), "m1_t0": round(float(m[0, 0]), 5),
            "sum_m_first4_t0": round(float(m[0, :min(4, Lc)].sum()), 5),
            "sum_m_first4_every_t1": [round(float(m[k, :min(4, Lc)].sum()), 5) for k in range(0, n_t, step)],
            "max_particle_hole_dev": float(np.max(np.abs(n[0] + n[1] - 1.0)))}
    return out


def c3_rows(n_t):
    """Rows of the 16-site-chain quench at full size (d = 130,873,600;
    columns of 91.6M and 147.2M states): ground state of H_ini, Phi on n_t
    grid times (t_k = 0.2 k, internal step 0.05), then the last row's step
    (iii) for the impurity's four blocks, timed."""
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c3()
    t0 = time.perf_counter()
    si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
    opts = kg.kg_opts_default(M=cfg["M"], dt_internal=cfg["dt_internal"], M_gs=40, tol_resid=1e-10,
                              max_restarts=400)
    E0, res, _ = si.ground_state(opts)
    K = kg.Keldysh(si, sf, cfg["orbitals"], cfg["dt"], n_t, opts)
    setup = time.perf_counter() - t0
    torch.cuda.synchronize()
    k = n_t - 1
    t1 = time.perf_counter()
    dl, dg = K.row(k)
    sec = time.perf_counter() - t1
    n_sub = int(round(cfg["dt"] / cfg["dt_internal"]))
    gsteps = 4 * k * n_sub
    plan = K.plan()
    K.close()
    return {"workload": "c3 16-site chain (7,7) d=130873600, row t_%d of step (iii): 4 columns (both spins, c and "
                        "c^dag; d=91.6M / 147.2M) x %d G-steps (dt_int=0.05, M=20)" % (k, k * n_sub),
            "setup_s": round(setup, 2), "seconds": round(sec, 2), "gsteps": gsteps,
            "gsteps_per_s": round(gsteps / sec, 3), "E0": E0, "gs_resid": res, "plan": plan,
            "sum_rule_dev": float(abs(1j * (dg[0, 0] - dl[0, 0]) - 1.0))}


def batched_vs_plain(n_inst, n_steps, plain_steps):
    """Equilibrium G_imp of the first n_inst star instances of the batched
    workload (256 instances, L in [6, 12], random fillings; dt = 0.05, M = 20,
    orbital (0, up)): n_steps steps through kg_green_equilibrium_batched, and
    plain_steps steps instance by instance through kg_green_equilibrium (the
    same steps repeat, so the two G-step rates compare).  Ground states are
    computed beforehand (untimed, the same for both); each path is run once
    untimed first (work lists, graphs, autotuning), then timed."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c4()
    models = cfg["models"][:n_inst]
    opts = kg.kg_opts_default(M=cfg["M"])
    secs = [kg.Sector(m) for m in models]
    ok = []
    for s in secs:
        try:
            s.ground_state(opts)
            ok.append(s)
        except kg.KGError:
            pass  # degenerate ground state: left out of both paths
    orbs, dt = cfg["orbitals"], cfg["dt"]
    def has_neighbour(s, dag):
        try:
            return s.neighbour_dim(0, dag) > 0
        except kg.KGError:
            return False  # full or empty up band: that part of G is zero

    cols = sum(sum(1 for dag in (False, True) if has_neighbour(s, dag)) for s in ok)
    gsteps = cols * n_steps
    kg.kg_green_equilibrium_batched([s.handle for s in ok], orbs, dt, min(n_steps, 4), opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gb, Lb, st = kg.kg_green_equilibrium_batched([s.handle for s in ok], orbs, dt, n_steps, opts)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    for s in ok[:4]:
        s.green_equilibrium(orbs, dt, 2, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    err = 0.0
    for i, s in enumerate(ok):
        g, l = s.green_equilibrium(orbs, dt, plain_steps, opts)
        err = max(err, float(np.max(np.abs(g - Gb[i, :plain_steps + 1]))),
                  float(np.max(np.abs(l - Lb[i, :plain_steps + 1]))))
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    plain_rate = cols * plain_steps / tp
    return {"workload": "first %d of 256 star-SIAM instances (L 6..12, random fillings, seed 20240501), "
                        "%d steps of dt=0.05 batched (%d per instance on the plain path), M=20, orbital (0,up), "
                        "G^> and G^<" % (n_inst, n_steps, plain_steps),
            "instances": len(ok), "gsteps": gsteps, "unit": "G-steps/s",
            "batched_value": round(gsteps / tb, 1), "plain_value": round(plain_rate, 1),
            "batched_s": round(tb, 3), "plain_s": round(tp, 3), "plain_steps": plain_steps,
            "speedup": round(gsteps / tb / plain_rate, 2), "max_abs_diff": err}


def lanczos_spectral(si, opts, n=100):
    """The conventional Lanczos Green's function (frequency domain) of the
    U = 8 ring's ground state: n = 100 Lanczos steps from c^dag_0|0> and
    c_0|0> (two columns, d = 731,808), continued fractions on 2001
    frequencies.  Ground state already computed (untimed)."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    omega = np.linspace(-10.0, 10.0, 2001)
    kg.kg_green_lanczos(si.handle, [(0, 0)], 8, omega[:3], 0.1, opts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gg, Gl, coef = kg.kg_green_lanczos(si.handle, [(0, 0)], n, omega, 0.1, opts)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    A = -(Gg[0] + Gl[0]).imag / np.pi
    return {"workload": "Lanczos G(omega) of the c2 ring ground state (U=8): n=%d steps from c^dag_0|0> and c_0|0> "
                        "(d=731808 each), eta=0.1, 2001 frequencies" % n,
            "seconds": round(t, 3), "lanczos_steps_per_s": round(2 * n / t, 1),
            "spectral_weight": round(float(np.trapezoid(A, omega) if hasattr(np, "trapezoid") else np.trapz(A, omega)), 4)}


def fine_grid_vs_plain(si, opts, n_steps=400, fine=8):
    """Equilibrium G_00(t) of the U = 8 ring on 401 times (dt = 0.05): one
    Krylov space per time step (M = 20) against one per `fine` times with the
    step exponential at several times (M = 40).  Ground state already
    computed (untimed); output times per second and the largest difference."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    o40 = kg.kg_opts_default(M=40, reorth=1, stream=opts.stream)
    kg.kg_green_equilibrium(si.handle, [(0, 0)], 0.05, 4, opts)  # warm-up
    kg.kg_green_equilibrium_fine(si.handle, [(0, 0)], 0.05, 2 * fine, fine, o40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gg, Gl = kg.kg_green_equilibrium(si.handle, [(0, 0)], 0.05, n_steps, opts)
    t1 = time.perf_counter()
    Fg, Fl = kg.kg_green_equilibrium_fine(si.handle, [(0, 0)], 0.05, n_steps, fine, o40)
    t2 = time.perf_counter()
    diff = float(max(np.max(np.abs(Fg - Gg)), np.max(np.abs(Fl - Gl))))
    return {"workload": "equilibrium G_00(t) of the c2 ring ground state (U=8), 401 times, dt=0.05",
            "plain_s": round(t1 - t0, 3), "fine_s": round(t2 - t1, 3), "fine": fine, "M_fine": 40,
            "speedup": round((t1 - t0) / (t2 - t1), 2), "max_abs_diff": diff}


def fourier_transform(fp64_tflops, n_t=100001, n_omega=4001):
    """The damped Fourier transform G(t) -> G(omega) at the sampling of the
    paper's Fig. 1 (dt' = 0.01 up to t_max = 1000, eta = 0.01): a particle
    and a hole series (synthetic sums of exponentials), 4001 frequencies on
    [-10, 10], host buffers in and out.  Counted as 8 flops (4 FP64 FMAs)
    per sample and frequency."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    rng = np.random.default_rng(5)
    dt = 0.01
    t = dt * np.arange(n_t)
    E = rng.uniform(-8.0, 8.0, size=(2, 8))
    A = rng.uniform(0.0, 1.0, size=(2, 8))
    G = -1j * np.einsum("sm,smk->sk", A / A.sum(1, keepdims=True), np.exp(-1j * E[:, :, None] * t))
    omega = np.linspace(-10.0, 10.0, n_omega)
    kg.kg_green_fourier(G[:, :2048], dt, omega[:512], 0.01)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = kg.kg_green_fourier(G, dt, omega, 0.01)
    sec = time.perf_counter() - t0
    tf = 8.0 * G.size * n_omega / sec / 1e12
    return {"workload": "damped Fourier transform, 2 series x %d samples (dt=0.01, t_max=1000, eta=0.01) onto %d "
                        "frequencies, host buffers" % (n_t, n_omega),
            "seconds": round(sec, 4), "tflops_fp64": round(tf, 3), "frac_fp64_measured": round(tf / fp64_tflops, 3),
            "spectral_weight": round(float(-np.trapezoid(F.imag, omega).sum() / np.pi / 2)
                                     if hasattr(np, "trapezoid") else float(-np.trapz(F.imag, omega).sum() / np.pi / 2), 4)}


def fig1_restarts(fs=(1, 100, 1000), n=100, dt=0.01, t_max=1000.0, eta=0.01):
    """Section 3, Fig. 1: the local spectral function of the half-filled L = 10
    Hubbard ring at U = 8 (particle-hole symmetric, omega > 0 shown) from
    G^R_00(t) = G^>(t) - G^<(t) on t <= 1000 at dt' = 0.01, by time-dependent
    Lanczos with n = 100 and f restarts, then the damped Fourier transform
    (eta = 0.01).  f = 1000 is the converged result; the paper reports that
    f = 1 (the conventional Lanczos function) stays non-negative while f = 100
    produces negative spectral weight.  Reported per f: time, the most
    negative A(omega), the negative weight, and the L1 distance to f = 1000."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    m = W.with_sector(W.hubbard_ring(10, 8.0, 5, 5), 5, 5)
    m["eps"] = np.full((2, 10), -4.0)  # particle-hole symmetric: eps = -U/2
    s = kg.Sector(m)
    s.ground_state()
    steps = int(round(t_max / dt))
    omega = np.linspace(0.0, 12.0, 2401)
    dw = omega[1] - omega[0]
    out, spectra = {}, {}
    for f in sorted(fs, reverse=True):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gg, Gl = s.green_restarted([(0, 0)], n, f, steps // f, dt)
        sec = time.perf_counter() - t0
        GR = (Gg - Gl)[:, 0, 0]
        A = -kg.kg_green_fourier(GR[None, :], dt, omega, eta)[0].imag / np.pi
        spectra[f] = A
        out["f=%d" % f] = {"seconds": round(sec, 2), "min_A": float(A.min()),
                           "negative_weight": float(-np.sum(np.minimum(A, 0.0)) * dw)}
    ref = spectra[max(fs)]
    for f in fs:
        out["f=%d" % f]["l1_to_f%d" % max(fs)] = float(np.sum(np.abs(spectra[f] - ref)) * dw)
    out["workload"] = ("L=10 ring U=8 half filling (d=63504), G_00 on t<=1000 at dt'=0.01, n=100, f restarts; "
                       "A(omega) for omega in [0,12] by the damped Fourier transform (eta=0.01)")
    return out


def adjoint_vs_fd():
    """Gradient of the bath-fitting loss sum_t |G_imp(t) - G_target(t)|^2 on the
    star L = 10 (5,5) workload (d = 63,504, 401 times, checkpoints every 20
    steps) with respect to the 19 parameters (eps_k, V_k, U): one adjoint
    (kg_green_equilibrium_vjp) against the 38 forward solves of central
    differences.  Each timed call builds its sector (ground state included)."""
    import numpy as np
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c5()
    orbs, dt, n = cfg["orbitals"], cfg["dt"], cfg["n_steps"]
    opts = kg.kg_opts_default(M=cfg["M"])
    Tg, Tl = kg.Sector(cfg["target"]).green_equilibrium(orbs, dt, n, opts)
    T = (Tg - Tl)[:, 0, 0]
    kg.Sector(cfg["start"]).green_equilibrium(orbs, dt, n, opts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gg, Gl = kg.Sector(cfg["start"]).green_equilibrium(orbs, dt, n, opts)
    tf = time.perf_counter() - t0
    r = 2.0 * ((Gg - Gl)[:, 0, 0] - T)
    dGg = np.zeros_like(Gg)
    dGl = np.zeros_like(Gl)
    dGg[:, 0, 0] = r
    dGl[:, 0, 0] = -r
    t0 = time.perf_counter()
    s = kg.Sector(cfg["start"])
    kg.kg_green_equilibrium_vjp(s.handle, 10, orbs, dt, n, dGg, dGl, opts, checkpoint=cfg["checkpoint"])
    tv = time.perf_counter() - t0
    return {"workload": "star SIAM L=10 (5,5) d=63504, 401 times dt=0.05, M=20, checkpoints every 20 steps, "
                        "19 fitted parameters", "forward_s": round(tf, 3), "vjp_s": round(tv, 3),
            "vjp_over_forward": round(tv / tf, 2), "fd_forwards": 38, "speedup_vs_fd": round(38 * tf / tv, 2)}


def cpu_baseline_sample(budget_s):
    """Oracle G-steps (exp(-iH dt) on one column of the N-1 sector) timed on the
    host cores until about budget_s seconds of work are done."""
    import oracle
    import workloads as W
    cfg = W.config_c2()
    sec = oracle.Sector(W.with_sector(cfg["fin"], 5, 6))
    x = W.random_state(sec.dim, 99)
    n, t0 = 0, time.perf_counter()
    while True:
        x = sec.propagate(x, -cfg["dt"])
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 200:
            break
    cores = oracle.num_threads()
    # the same oracle on one core, a shorter sample
    oracle.set_num_threads(1)
    try:
        n1, t1 = 0, time.perf_counter()
        while True:
            x = sec.propagate(x, -cfg["dt"])
            n1 += 1
            el1 = time.perf_counter() - t1
            if el1 > budget_s / 2 or n1 >= 50:
                break
    finally:
        oracle.set_num_threads(cores)
    return {"value": round(n / el, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d oracle G-steps (Chebyshev exp(+iH*0.05) of one c2 N-1 column, d=%d) in %.1f s"
                      % (n, sec.dim, el),
            "single_thread": {"value": round(n1 / el1, 4), "unit": UNIT, "cores": 1,
                              "sample": "%d oracle G-steps of the same column on one thread in %.1f s" % (n1, el1)}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W
    cfg = W.config_c2()
    sec = oracle.Sector(W.with_sector(cfg["fin"], 5, 6))
    x = W.random_state(sec.dim, 99)
    per_step = max(1, args.ref_gsteps)
    for _ in range(args.warmup):
        x = sec.propagate(x, -cfg["dt"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            x = sec.propagate(x, -cfg["dt"])
    el = time.perf_counter() - t0
    value = args.steps * per_step / el
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": row_workload(cfg["n_t"] - 1), "column_dim": sec.dim, "M": cfg["M"], "reorth": 1},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "bounded sample of that row: %d oracle G-steps (Chebyshev exp(+iH*0.05) of one "
                                   "N-1 column, d=%d) per step" % (per_step, sec.dim)},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ncu_case(args):
    """Small case for ncu captures: one Keldysh row of the c2 quench restricted
    to --ncu-orbitals orbitals (default 6: two batches of 6 columns of the
    N-1 / N+1 sectors, d = 731,808, 1.5 GB of Krylov basis per batch, more
    than the L2; 12 gives the benchmark's batch width), backward by 2 Krylov
    steps with the benchmark's options.  The row runs inside the NVTX range
    "row" so that a capture can skip the set-up."""
    import torch

    import paper_1109_1205_gb300 as kg
    import workloads as W
    cfg = W.config_c2()
    opts = kg.kg_opts_default(M=cfg["M"], reorth=1, schedule=args.schedule)
    if args.ncu_hpsi:
        # the standalone H*psi on a column of the N-1 sector, three calls
        # inside the NVTX range "hpsi"
        nb = kg.Sector(W.with_sector(cfg["fin"], 5, 6))
        x = torch.randn(nb.dim, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("hpsi")
        for _ in range(3):
            nb.hpsi(x, y, torch.cuda.current_stream())
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"ncu_case": "standalone H*psi, d=%d" % nb.dim, "launches": kg.kg_launch_count()}))
        return
    si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
    si.ground_state(opts)
    K = kg.Keldysh(si, sf, cfg["orbitals"][:args.ncu_orbitals], cfg["dt"], 3, opts)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("row")
    Gl, Gg = K.row(2)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"ncu_case": "c2 row t_2, %d orbitals" % args.ncu_orbitals, "d": sf.dim,
                      "launches": kg.kg_launch_count(),
                      "G_les_00": [float(Gl[0, 0].real), float(Gl[0, 0].imag)]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-gsteps", type=int, default=4)
    ap.add_argument("--ncu-case", action="store_true", help="small case for full ncu captures")
    ap.add_argument("--ncu-orbitals", type=int, default=6, help="orbitals of the ncu case (12 = the full row)")
    ap.add_argument("--ncu-hpsi", action="store_true", help="ncu case: the standalone H*psi instead of a row")
    ap.add_argument("--schedule", type=int, default=0, help="kg_opts.schedule of the ncu case")
    ap.add_argument("--fig1-case", action="store_true", help="only the restarted-Lanczos comparison of Fig. 1")
    ap.add_argument("--fourier-case", action="store_true",
                    help="only the damped Fourier transform extra (for ncu captures of k_fourier)")
    ap.add_argument("--driven-case", action="store_true", help="only the driven-H(t) extra on the c2 ring")
    ap.add_argument("--necpt-case", action="store_true", help="only the NE-CPT extra, clusters of 4, 6 and 8 sites")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint comparisons")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=400)
    ap.add_argument("--plain-steps", type=int, default=100)
    ap.add_argument("--no-c2-full", action="store_true", help="skip the whole-grid c2 time to solution")
    ap.add_argument("--c3", action="store_true", help="also time a row of the 16-site chain at full size")
    ap.add_argument("--c3-nt", type=int, default=3, help="grid times of the c3 row extra (row n_t - 1 is timed)")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.fig1_case:
        print(json.dumps({"fig1_case": fig1_restarts()}))
        return
    if args.driven_case:
        import paper_1109_1205_gb300 as kg
        import workloads as W
        cfg = W.config_c2()
        opts = kg.kg_opts_default(M=cfg["M"], reorth=1)
        si, sf = kg.Sector(cfg["ini"]), kg.Sector(cfg["fin"])
        si.ground_state(opts)
        print(json.dumps({"driven_case": driven_vs_quench(si, sf, opts), "four_time": four_time(si, sf, opts)}))
        return
    if args.necpt_case:
        print(json.dumps({"necpt_case": necpt_fig5(sizes=(4, 6, 8))}))
        return
    if args.fourier_case:
        import paper_1109_1205_gb300 as kg
        print(json.dumps({"fourier_case": fourier_transform(kg.kg_probe_fp64(None))}))
        return
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
